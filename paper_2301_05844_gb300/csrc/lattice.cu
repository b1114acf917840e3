// bbp_create_lattice / bbp_set_tensors / bbp_sweep / bbp_destroy and the message
// inspection calls.  The sweep of Eq. 1 is planned here (see engine.cu for the fit).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bbp.h"
#include "bbp_internal.h"
#include "engine.h"
#include "lattice.h"

using namespace bbp;

// Pinned read-back words come from slabs that live as long as the process: freeing
// page-locked memory synchronises the whole device, which a lattice destroyed while
// others run must not do.
static std::mutex g_pin_mu;
static std::vector<PinnedWords*> g_pin_free;

static PinnedWords* pinned_get() {
    std::lock_guard<std::mutex> g(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int SLAB = 64;
        PinnedWords* slab = nullptr;
        if (cudaMallocHost((void**)&slab, SLAB * sizeof(PinnedWords)) != cudaSuccess) return nullptr;
        for (int i = SLAB - 1; i >= 0; --i) g_pin_free.push_back(slab + i);
    }
    PinnedWords* p = g_pin_free.back();
    g_pin_free.pop_back();
    *p = PinnedWords{};
    return p;
}

static void pinned_put(PinnedWords* p) {
    std::lock_guard<std::mutex> g(g_pin_mu);
    g_pin_free.push_back(p);
}

#define CKR(expr)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) return fail(BBP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ geometry
int bbp_lattice::tensor_index(int r, int c) const {
    if (desc.boundary == BBP_OBC) return r * desc.Lx + c;
    // block site (r, c) of a shifted partition is lattice site (r + shift_y, c + shift_x)
    return ((r + desc.shift_y) % desc.Ly) * desc.Lx + ((c + desc.shift_x) % desc.Lx);
}

std::array<int, 4> bbp_lattice::site_dims(int r, int c) const {
    const int D = desc.D;
    if (desc.boundary != BBP_OBC) return {D, D, D, D};
    return {r == 0 ? 1 : D, c == 0 ? 1 : D, r == desc.Ly - 1 ? 1 : D, c == desc.Lx - 1 ? 1 : D};
}

int bbp_lattice::neighbour(int blk, int dir) const {
    if (desc.boundary != BBP_OBC) return blk;
    const int R = blk / nbx, C = blk % nbx;
    int R2 = R, C2 = C;
    if (dir == DIR_LEFT) C2--;
    if (dir == DIR_RIGHT) C2++;
    if (dir == DIR_UP) R2--;
    if (dir == DIR_DOWN) R2++;
    if (R2 < 0 || R2 >= nby || C2 < 0 || C2 >= nbx) return -1;
    return R2 * nbx + C2;
}

void bbp_lattice::block_origin(int blk, int& r0, int& c0) const {
    r0 = ys[blk / nbx];
    c0 = xs[blk % nbx];
}

void bbp_lattice::block_size(int blk, int& h, int& w) const {
    const int R = blk / nbx, C = blk % nbx;
    h = ys[R + 1] - ys[R];
    w = xs[C + 1] - xs[C];
}

int bbp_lattice::block_of(int r, int c) const {
    const int R = (int)(std::upper_bound(ys.begin(), ys.end(), r) - ys.begin()) - 1;
    const int C = (int)(std::upper_bound(xs.begin(), xs.end(), c) - xs.begin()) - 1;
    return R * nbx + C;
}

View3 bbp_lattice::msg_site(int it, int s, bool cur) const {
    const Item& I = items[it];
    return contiguous3((cur ? msg_cur : msg_new) + I.region_off + I.site_off[s], I.mb[s], K, I.mb[s + 1]);
}

static View3 one3(size_t one_off) {
    View3 v;
    v.off = one_off;
    return v;  // 1x1x1, zero strides
}

std::vector<View3> bbp_lattice::incoming(int blk, int dir) const {
    int bh, bw;
    block_size(blk, bh, bw);
    const int nsite = (dir == DIR_LEFT || dir == DIR_RIGHT) ? bh : bw;
    std::vector<View3> v;
    const int nb = neighbour(blk, dir);
    if (nb < 0) {
        for (int i = 0; i < nsite; ++i) v.push_back(one3(one_off));
        return v;
    }
    const int it = item_of[nb * 4 + opposite(dir)];
    for (int i = 0; i < nsite; ++i) v.push_back(msg_site(it, i, true));
    return v;
}

// MPO view O[w,p,q,w2] = E'[u', r', l', d'] of tensor t in the frame where `dir` is LEFT.
View4 bbp_lattice::E_view(int t, int dir) const {
    int map[4] = {0, 1, 2, 3};  // frame leg (u',l',d',r') -> original leg (u,l,d,r)
    if (dir == DIR_RIGHT) {
        map[0] = 0; map[1] = 3; map[2] = 2; map[3] = 1;
    } else if (dir == DIR_UP) {
        map[0] = 1; map[1] = 0; map[2] = 3; map[3] = 2;
    } else if (dir == DIR_DOWN) {
        map[0] = 1; map[1] = 2; map[2] = 3; map[3] = 0;
    }
    const auto& dd = tdims[t];
    int Kd[4];
    for (int i = 0; i < 4; ++i) Kd[i] = single ? dd[i] : dd[i] * dd[i];
    long long st[4] = {(long long)Kd[1] * Kd[2] * Kd[3], (long long)Kd[2] * Kd[3], Kd[3], 1};
    View4 o;
    o.off = E_off[t];
    o.w = Kd[map[0]]; o.sw = st[map[0]];
    o.p = Kd[map[3]]; o.sp = st[map[3]];
    o.q = Kd[map[1]]; o.sq = st[map[1]];
    o.w2 = Kd[map[2]]; o.sw2 = st[map[2]];
    return o;
}

// Frame site (rf, cf) of a bh x bw region at (r0, c0) rotated so that `dir` is LEFT.
View4 bbp_lattice::frame_E(int dir, int r0, int c0, int bh, int bw, int rf, int cf, int* tensor) const {
    int r = rf, c = cf;
    if (dir == DIR_RIGHT) {
        c = bw - 1 - cf;
    } else if (dir == DIR_UP) {
        r = cf; c = rf;
    } else if (dir == DIR_DOWN) {
        r = bh - 1 - cf; c = rf;
    }
    const int t = tensor_index(r0 + r, c0 + c);
    if (tensor) *tensor = t;
    return E_view(t, dir);
}

static std::vector<View3> reversed(const std::vector<View3>& m) {
    std::vector<View3> r;
    for (int i = (int)m.size() - 1; i >= 0; --i) r.push_back(reversed3(m[i]));
    return r;
}

FrameMsgs bbp_lattice::frame_msgs(int dir, const std::vector<View3> in[4]) const {
    FrameMsgs f;
    if (dir == DIR_LEFT) {
        f.T = in[DIR_UP]; f.R = in[DIR_RIGHT]; f.B = in[DIR_DOWN];
    } else if (dir == DIR_RIGHT) {
        f.T = reversed(in[DIR_UP]); f.R = in[DIR_LEFT]; f.B = reversed(in[DIR_DOWN]);
    } else if (dir == DIR_UP) {
        f.T = in[DIR_LEFT]; f.R = in[DIR_DOWN]; f.B = in[DIR_RIGHT];
    } else {
        f.T = reversed(in[DIR_LEFT]); f.R = in[DIR_UP]; f.B = reversed(in[DIR_RIGHT]);
    }
    return f;
}

namespace bbp {
// Column MPO of frame column c: [top message site, E'(0,c) .. E'(H-1,c), bottom site].
std::vector<View4> column_mpo(const bbp_lattice* L, int dir, int r0, int c0, int bh, int bw, const FrameMsgs& fm, int c) {
    const int H = (dir == DIR_LEFT || dir == DIR_RIGHT) ? bh : bw;
    std::vector<View4> O;
    const View3& t = fm.T[c];
    View4 top;
    top.off = t.off; top.w = 1; top.p = t.b; top.q = t.a; top.w2 = t.k;
    top.sw = 0; top.sp = t.sb; top.sq = t.sa; top.sw2 = t.sk;
    O.push_back(top);
    for (int r = 0; r < H; ++r) O.push_back(L->frame_E(dir, r0, c0, bh, bw, r, c));
    const View3& b = fm.B[c];
    View4 bot;
    bot.off = b.off; bot.w = b.k; bot.p = b.b; bot.q = b.a; bot.w2 = 1;
    bot.sw = b.sk; bot.sp = b.sb; bot.sq = b.sa; bot.sw2 = 0;
    O.push_back(bot);
    return O;
}

// Lay out and emit the fits of a set of column sweeps.  Each sweep i has a frame
// (dir, region), its frame messages and chi; `keep` keeps every column's Y (read-out),
// otherwise two ping-pong buffers are used.  Fills sweeps[i].fits.
int plan_column_sweeps(bbp_lattice* L, Program& pr, std::vector<ColumnSweep>& cs, int max_sweeps, double fit_tol,
                       bool rand_uses_sweep, bool mixed, bool warm) {
    const int ss = L->ss;
    const MixCtx& cx = L->cx;
    auto pad = [&](long long x) { return padded(cx, x); };
    auto lp_alloc = [&](size_t elems) { return pr.lp_alloc(elems, cx.esz, cx.x3); };
    auto elem_alloc = [&](size_t elems) { return pr.arena_alloc(elems * (size_t)ss) / (size_t)ss; };
    for (auto& s : cs) {
        const int H = (s.dir == DIR_LEFT || s.dir == DIR_RIGHT) ? s.bh : s.bw;
        const int W = (s.dir == DIR_LEFT || s.dir == DIR_RIGHT) ? s.bw : s.bh;
        const int n = H + 2;
        s.H = H;
        s.W = W;
        // shapes per column
        std::vector<std::vector<View4>> Os(W);
        std::vector<std::vector<int>> q(W), yb(W);
        for (int c = 0; c < W; ++c) {
            Os[c] = column_mpo(L, s.dir, s.r0, s.c0, s.bh, s.bw, s.fm, c);
            for (auto& o : Os[c]) q[c].push_back(o.q);
            yb[c] = bond_caps(q[c], s.chi);
        }
        // capacities
        const int nbuf = s.keep ? W : 2;
        std::vector<size_t> ycap(n, 1), acap(n + 1, 1);
        size_t t1cap = 1, t2cap = 1, ytcap = 1, qrcap = 1;
        for (int c = 0; c < W; ++c) {
            for (int i = 0; i < n; ++i) ycap[i] = std::max(ycap[i], (size_t)yb[c][i] * q[c][i] * yb[c][i + 1]);
            for (int i = 0; i < n; ++i) {
                const View4& o = Os[c][i];
                const int y = yb[c][i], y2 = yb[c][i + 1];
                // X dims of this column
                int x, x2;
                if (c == W - 1) {
                    x = (i == 0 || i == n - 1) ? 1 : s.fm.R[i - 1].a;
                    x2 = (i == 0 || i == n - 1) ? 1 : s.fm.R[i - 1].b;
                    if (i == 0) x2 = 1;
                } else {
                    x = yb[c + 1][i];
                    x2 = yb[c + 1][i + 1];
                }
                const size_t p = o.p, w = o.w, w2 = o.w2, qq = o.q;
                acap[i + 1] = std::max(acap[i + 1], (size_t)y2 * w2 * x2);
                acap[i] = std::max(acap[i], (size_t)y * w * x);
                t1cap = std::max({t1cap, (size_t)y * w * p * x2, (size_t)x * p * y2 * w2});
                t2cap = std::max({t2cap, (size_t)y * x2 * qq * w2, (size_t)x * y2 * w * qq});
                ytcap = std::max(ytcap, (size_t)y * qq * y2);
                qrcap = std::max(qrcap, 2 * (size_t)y * qq * y2);
            }
        }
        std::vector<std::vector<size_t>> ybuf(nbuf, std::vector<size_t>(n));
        for (int bi = 0; bi < nbuf; ++bi)
            for (int i = 0; i < n; ++i) ybuf[bi][i] = elem_alloc(ycap[i]);
        std::vector<size_t> A(n + 1), B(n + 1);
        A[0] = L->one_off;
        B[n] = L->one_off;
        for (int i = 1; i <= n; ++i) A[i] = elem_alloc(acap[i]);
        for (int i = 0; i < n; ++i) B[i] = elem_alloc(acap[i]);
        const size_t T1 = elem_alloc(t1cap), T2 = elem_alloc(t2cap), Yt = elem_alloc(ytcap), qrw = elem_alloc(qrcap);
        const size_t losses = pr.arena_alloc(sizeof(double) * (size_t)max_sweeps * 2 * (n - 1));
        const size_t active = pr.arena_alloc(sizeof(int));
        s.fits.assign(W, FitSpec());
        for (int c = W - 1; c >= 0; --c) {
            FitSpec& f = s.fits[c];
            f.O = Os[c];
            f.ybond = yb[c];
            const int bi = s.keep ? c : (c % 2);
            f.Y = ybuf[bi];
            if (c == W - 1) {
                f.X.push_back(one3(L->one_off));
                for (auto& v : s.fm.R) f.X.push_back(v);
                f.X.push_back(one3(L->one_off));
            } else {
                const int pb = s.keep ? c + 1 : ((c + 1) % 2);
                for (int i = 0; i < n; ++i)
                    f.X.push_back(contiguous3(ybuf[pb][i], yb[c + 1][i], q[c + 1][i], yb[c + 1][i + 1]));
            }
            for (int i = 0; i < n; ++i)
                if (f.X[i].k != f.O[i].p) return fail(BBP_ERR_INVALID, "internal: column MPS / MPO leg mismatch");
            f.Aenv = A;
            f.Benv = B;
            f.T1 = T1; f.T2 = T2; f.Yt = Yt; f.qrw = qrw;
            f.losses = losses;
            f.active = active;
            f.counter = pr.arena_alloc(sizeof(int));
            f.stream = stream_id(s.tag, s.outer, s.msg, (uint64_t)c, 0);
            if (s.warm_from) {
                const FitSpec& g = (*s.warm_from)[c];
                if (g.ybond != f.ybond || g.n() != f.n()) return fail(BBP_ERR_INVALID, "internal: warm source shape");
                f.warm = true;
            }
        }
        if (!mixed) continue;
        // low-precision operand buffers, sized for every column of this sweep
        std::vector<size_t> cxl(n, 1), cxr(n, 1), cys(n, 1), cyt(n, 1), cer(n + 1, 1), cek(n + 1, 1), cocl(2, 1), cocr(2, 1);
        size_t ct1 = 1, ct2a = 1, ct2b = 1, cytf = 1;
        for (int c = 0; c < W; ++c) {
            const FitSpec& f = s.fits[c];
            for (int i = 0; i < n; ++i) {
                const long long y = f.ybond[i], y2 = f.ybond[i + 1], x = f.X[i].a, x2 = f.X[i].b, p = f.X[i].k;
                const long long w = f.O[i].w, w2 = f.O[i].w2, q = f.O[i].q;
                cxl[i] = std::max(cxl[i], (size_t)(p * x2 * pad(x)));
                cxr[i] = std::max(cxr[i], (size_t)(x * p * pad(x2)));
                cys[i] = std::max(cys[i], (size_t)(y * pad(q * y2)));
                cyt[i] = std::max(cyt[i], (size_t)(y2 * pad(y * q)));
                cer[i] = std::max(cer[i], (size_t)(y * w * pad(x)));
                cek[i] = std::max(cek[i], (size_t)(y * pad(w * x)));
                cer[i + 1] = std::max(cer[i + 1], (size_t)(y2 * w2 * pad(x2)));
                cek[i + 1] = std::max(cek[i + 1], (size_t)(y2 * pad(w2 * x2)));
                ct1 = std::max({ct1, (size_t)(y * x2 * pad(w * p)), (size_t)(x * y2 * pad(p * w2))});
                ct2a = std::max({ct2a, (size_t)(y * q * pad(w2 * x2)), (size_t)(q * y2 * pad(w * x))});
                ct2b = std::max({ct2b, (size_t)(w2 * x2 * pad(y * q)), (size_t)(w * x * pad(q * y2))});
                cytf = std::max(cytf, (size_t)(y * q * y2));
                if (i == 0 || i == n - 1) {
                    const int k = i == 0 ? 0 : 1;
                    cocl[k] = std::max(cocl[k], (size_t)(q * w2 * pad(w * p)));
                    cocr[k] = std::max(cocr[k], (size_t)(w * q * pad(p * w2)));
                }
            }
        }
        MixBufs mb;
        for (int i = 0; i < n; ++i) {
            mb.XL.push_back(lp_alloc(cxl[i]));
            mb.XR.push_back(lp_alloc(cxr[i]));
            mb.YS.push_back(lp_alloc(cys[i]));
            mb.YT.push_back(lp_alloc(cyt[i]));
        }
        for (int i = 0; i <= n; ++i) {
            const bool edgeA = i == 0, edgeB = i == n;
            mb.AR.push_back(edgeA ? L->one_lp : lp_alloc(cer[i]));
            mb.AK.push_back(edgeA ? L->one_lp : lp_alloc(cek[i]));
            mb.BR.push_back(edgeB ? L->one_lp_b : lp_alloc(cer[i]));
            mb.BK.push_back(edgeB ? L->one_lp_b : lp_alloc(cek[i]));
        }
        mb.T1 = lp_alloc(ct1);
        mb.T2a = lp_alloc(ct2a);
        mb.T2b = lp_alloc(ct2b);
        mb.Ytf = pr.arena_alloc(cytf * sizeof(float));
        const size_t ocl[2] = {lp_alloc(cocl[0]), lp_alloc(cocl[1])}, ocr[2] = {lp_alloc(cocr[0]), lp_alloc(cocr[1])};
        for (int c = 0; c < W; ++c) {
            FitSpec& f = s.fits[c];
            f.mixed = true;
            f.mx = mb;
            f.mx.OL.assign(n, 0);
            f.mx.OR.assign(n, 0);
            f.mx.OL[0] = ocl[0]; f.mx.OR[0] = ocr[0];
            f.mx.OL[n - 1] = ocl[1]; f.mx.OR[n - 1] = ocr[1];
            for (int r = 0; r < H; ++r) {
                int t = 0;
                L->frame_E(s.dir, s.r0, s.c0, s.bh, s.bw, r, c, &t);
                f.mx.OL[r + 1] = L->EL_off[t][s.dir];
                f.mx.OR[r + 1] = L->ER_off[t][s.dir];
            }
        }
    }
    // emit, lockstep over column steps
    int Wmax = 0;
    for (auto& s : cs) Wmax = std::max(Wmax, s.W);
    for (int k = 0; k < Wmax; ++k) {
        std::vector<FitSpec*> group;
        std::vector<RelayoutTask> warm_copy;  // FP64 copies of the warm sources' fitted MPS
        for (auto& s : cs) {
            const int c = s.W - 1 - k;
            if (c < 0) continue;
            group.push_back(&s.fits[c]);
            if (!s.warm_from) continue;
            const FitSpec& g = (*s.warm_from)[c];
            const FitSpec& f = s.fits[c];
            for (int i = 0; i < f.n(); ++i) {
                RelayoutTask r{};
                r.src = P(g.Y[i] * (size_t)ss);
                r.dst = P(f.Y[i] * (size_t)ss);
                r.src_kind = 0;
                r.dst_kind = 0;
                r.d[0] = f.ybond[i] * f.O[i].q * f.ybond[i + 1];
                r.d[1] = r.d[2] = r.d[3] = 1;
                r.ss[0] = 1;
                r.ds[0] = 1;
                if (L->cplx) {  // complex scalars as pairs of doubles
                    r.d[0] *= 2;
                }
                warm_copy.push_back(r);
            }
        }
        pr.rel_step(warm_copy);
        if (!mixed) {
            emit_fits(pr, ss, group, max_sweeps, fit_tol, warm, rand_uses_sweep);
            continue;
        }
        // low-precision copies of this column's X (messages or the previous column's Y,
        // both FP64) and of its two corner MPO sites (message sites)
        std::vector<RelayoutTask> rt;
        auto rel3 = [&](const View3& v, size_t dst, int order) {
            RelayoutTask r{};
            r.src = P(v.off * (size_t)ss);
            r.dst = P(dst);
            r.src_kind = 0;
            r.dst_kind = cx.lpk;
            if (order == 0) {  // XL[x2][p][pad x]  (B operand of K2)
                r.d[0] = v.b; r.d[1] = v.k; r.d[2] = v.a; r.d[3] = 1;
                r.ss[0] = v.sb; r.ss[1] = v.sk; r.ss[2] = v.sa;
                r.ds[0] = (long long)v.k * pad(v.a); r.ds[1] = pad(v.a); r.ds[2] = 1;
                r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? pr.plane_of(dst) : 0;
            } else {  // XR[x][p][pad x2]  (A operand of K2r)
                r.d[0] = v.a; r.d[1] = v.k; r.d[2] = v.b; r.d[3] = 1;
                r.ss[0] = v.sa; r.ss[1] = v.sk; r.ss[2] = v.sb;
                r.ds[0] = (long long)v.k * pad(v.b); r.ds[1] = pad(v.b); r.ds[2] = 1;
                r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? pr.plane_of(dst) : 0;
            }
            rt.push_back(r);
        };
        auto rel4 = [&](const View4& o, size_t dst, int order) {
            RelayoutTask r{};
            r.src = P(o.off * (size_t)ss);
            r.dst = P(dst);
            r.src_kind = 0;
            r.dst_kind = cx.lpk;
            if (order == 0) {  // OL[w2][q][pad(w p)]
                r.d[0] = o.w2; r.d[1] = o.q; r.d[2] = o.w; r.d[3] = o.p;
                r.ss[0] = o.sw2; r.ss[1] = o.sq; r.ss[2] = o.sw; r.ss[3] = o.sp;
                r.ds[0] = (long long)o.q * pad((long long)o.w * o.p); r.ds[1] = pad((long long)o.w * o.p); r.ds[2] = o.p; r.ds[3] = 1;
                r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? pr.plane_of(dst) : 0;  // B operand of K3
            } else {  // OR[w][q][pad(p w2)]
                r.d[0] = o.w; r.d[1] = o.q; r.d[2] = o.p; r.d[3] = o.w2;
                r.ss[0] = o.sw; r.ss[1] = o.sq; r.ss[2] = o.sp; r.ss[3] = o.sw2;
                r.ds[0] = (long long)o.q * pad((long long)o.p * o.w2); r.ds[1] = pad((long long)o.p * o.w2); r.ds[2] = o.w2; r.ds[3] = 1;
                r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? pr.plane_of(dst) : 0;  // B operand of K3r
            }
            rt.push_back(r);
        };
        for (auto* f : group) {
            const int n = f->n();
            for (int i = 0; i < n; ++i) {
                rel3(f->X[i], f->mx.XL[i], 0);
                rel3(f->X[i], f->mx.XR[i], 1);
            }
            rel4(f->O[0], f->mx.OL[0], 0);
            rel4(f->O[0], f->mx.OR[0], 1);
            rel4(f->O[n - 1], f->mx.OL[n - 1], 0);
            rel4(f->O[n - 1], f->mx.OR[n - 1], 1);
        }
        pr.rel_step(rt);
        emit_fits_mixed(pr, cx, group, max_sweeps, fit_tol, warm, rand_uses_sweep);
    }
    return BBP_OK;
}
}  // namespace bbp

// Lower bound on the zip-up fit tolerance of a precision.  The stop rule compares
// std/|mean| of a sweep's losses (App. A); a loss computed from plain TF32 / BF16
// contractions carries relative noise near 1e-3 / 1e-2, below which the rule never fires,
// so those paths raise the tolerance to 3e-3 / 3e-2.  The split paths (TF32X3, BF16X3)
// accumulate products of long contractions in FP32 (K up to 3 x 2400 at D=5, chi=96), whose
// rounding leaves relative loss noise of order 2^-24 sqrt(K), about 5e-6 there: both take
// 3e-5 (at 1e-6, and for TF32X3 at 1e-5, some fits of the D=5, chi=96 lattices ran to the
// sweep cap).
double bbp::fit_tol_floor(int prec) {
    switch (prec) {
        case BBP_PREC_TF32: return 3e-3;
        case BBP_PREC_BF16: return 3e-2;
        case BBP_PREC_TF32X3:
        case BBP_PREC_BF16X3: return 3e-5;
        default: return 0.0;
    }
}

// ------------------------------------------------------------------ plan one sweep
static int plan_sweep(bbp_lattice* L) {
    Program& pr = L->sweep;
    pr.cplx = L->cplx;
    const int ss = L->ss;
    // the sweep counter first: warm-started fits read it
    const size_t sweepctr = pr.arena_alloc(sizeof(int));
    pr.warm_ctr_off = sweepctr;
    // the column sweep of every item
    std::vector<ColumnSweep> cs;
    for (int it = 0; it < (int)L->items.size(); ++it) {
        const Item& I = L->items[it];
        std::vector<View3> in[4];
        for (int d = 0; d < 4; ++d) in[d] = L->incoming(I.block, d);
        ColumnSweep s;
        s.dir = I.dir;
        L->block_origin(I.block, s.r0, s.c0);
        L->block_size(I.block, s.bh, s.bw);
        s.fm = L->frame_msgs(I.dir, in);
        s.chi = L->desc.chi;
        s.keep = L->desc.warm_start != 0;  // per-column Y buffers persist across sweeps
        s.tag = 0;
        s.outer = 0;
        s.msg = (uint64_t)I.msgid;
        cs.push_back(s);
    }
    double fit_tol = std::max(L->desc.fit_tol, fit_tol_floor(L->desc.prec));
    int rc = plan_column_sweeps(L, pr, cs, L->desc.fit_max_sweeps, fit_tol, true, L->mixed,
                                L->desc.warm_start != 0);
    if (rc) return rc;
    for (int it = 0; it < (int)L->items.size(); ++it) L->items[it].fits = cs[it].fits;
    // message assembly from the final column MPS (column 0)
    std::vector<OverlapSpec> ov;
    std::vector<AssembleTask> at;
    std::vector<NormTask> nt;
    auto elem_alloc = [&](size_t elems) { return pr.arena_alloc(elems * (size_t)ss) / (size_t)ss; };
    const int K = L->K;
    for (int it = 0; it < (int)L->items.size(); ++it) {
        const Item& I = L->items[it];
        const FitSpec& f = I.fits[0];
        const int n = f.n();
        if (I.b > 16) return fail(BBP_ERR_INVALID, "block edge longer than 16 sites");
        AssembleTask a{};
        a.nsites = I.b;
        for (int s = 0; s < I.b; ++s) {
            const View3 dst = L->msg_site(it, s, false);
            if (f.ybond[s + 1] != dst.a || f.O[s + 1].q != dst.k || f.ybond[s + 2] != dst.b)
                return fail(BBP_ERR_INVALID, "internal: message shape mismatch");
            a.src[s] = P(f.Y[s + 1] * ss);
            a.dst[s] = P(dst.off * ss);
            a.size[s] = (long long)dst.a * dst.k * dst.b;
        }
        a.corner0 = P(f.Y[0] * ss);
        a.corner1 = P(f.Y[n - 1] * ss);
        at.push_back(a);
        // overlap chains <m|m> and <m|m_old>
        int amax = 1;
        for (int v : I.mb) amax = std::max(amax, v);
        for (int which = 0; which < 2; ++which) {
            OverlapSpec o;
            for (int s = 0; s < I.b; ++s) {
                o.M.push_back(L->msg_site(it, s, false));
                o.N.push_back(L->msg_site(it, s, which == 1));
            }
            o.one = L->one_off;
            o.E[0] = elem_alloc((size_t)amax * amax);
            o.E[1] = elem_alloc((size_t)amax * amax);
            o.T = elem_alloc((size_t)amax * K * amax);
            o.result = elem_alloc(1);
            ov.push_back(o);
        }
        NormTask nm{};
        const View3 s0 = L->msg_site(it, 0, false);
        nm.site0 = P(s0.off * ss);
        nm.size0 = (long long)s0.a * s0.k * s0.b;
        nm.nsites = I.b;
        nm.D = L->desc.D;
        nm.ones = L->single ? 1 : 0;
        for (int s = 0; s < I.b; ++s) {
            const View3 v = L->msg_site(it, s, false);
            nm.sites[s] = P(v.off * ss);
            nm.a[s] = v.a;
            nm.k[s] = v.k;
            nm.b[s] = v.b;
        }
        nm.mm = P(ov[ov.size() - 2].result * ss);
        nm.mo = P(ov[ov.size() - 1].result * ss);
        nm.resid = (double*)P((size_t)it * sizeof(double) + 1);  // patched below
        nt.push_back(nm);
    }
    {
        Step s;
        s.kind = ST_ASM;
        s.first = pr.asmb.size();
        s.count = (int)at.size();
        pr.asmb.insert(pr.asmb.end(), at.begin(), at.end());
        pr.steps.push_back(s);
    }
    emit_overlaps(pr, ss, ov);
    const size_t resid = pr.arena_alloc(sizeof(double) * std::max<size_t>(1, L->items.size()));
    const size_t residual = pr.arena_alloc(sizeof(double));
    const size_t status = pr.arena_alloc(sizeof(int));
    for (int it = 0; it < (int)nt.size(); ++it) {
        nt[it].resid = (double*)P(resid + (size_t)it * sizeof(double));
        nt[it].status = (int*)P(status);
    }
    {
        Step s;
        s.kind = ST_NORM;
        s.first = pr.nrm.size();
        s.count = (int)nt.size();
        pr.nrm.insert(pr.nrm.end(), nt.begin(), nt.end());
        pr.steps.push_back(s);
    }
    pr.simple(ST_MEAN, P(resid), P(residual), (long long)L->items.size(), 0);
    pr.simple(ST_COPY, P(L->msg_new * ss), P(L->msg_cur * ss), (long long)(L->msg_elems * ss), 0);
    pr.simple(ST_INC, P(sweepctr), nullptr, 1, 0);
    L->d_resid_terms = (double*)(uintptr_t)resid;
    L->d_residual = (double*)(uintptr_t)residual;
    L->d_status = (int*)(uintptr_t)status;
    L->d_sweep = (int*)(uintptr_t)sweepctr;
    return BBP_OK;
}

// ------------------------------------------------------------------ C ABI
// CUDA events and stream-ordered device allocations released on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};
struct AsyncBuffer {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    explicit AsyncBuffer(cudaStream_t st) : s(st) {}
    ~AsyncBuffer() {
        if (p) cudaFreeAsync(p, s);
    }
};

extern "C" {

const char* bbp_last_error(void) { return bbp::g_err.c_str(); }

static int validate(const bbp_lattice_desc* d) {
    if (!d) return fail(BBP_ERR_INVALID, "desc is NULL");
    if (d->Lx < 1 || d->Ly < 1 || d->d < 1 || d->D < 1 || d->bx < 1 || d->by < 1 || d->chi < 1)
        return fail(BBP_ERR_INVALID, "dimensions must be positive");
    if (d->boundary != BBP_OBC && d->boundary != BBP_INFINITE) return fail(BBP_ERR_INVALID, "unknown boundary");
    if (d->boundary == BBP_OBC && (d->Lx % d->bx || d->Ly % d->by))
        return fail(BBP_ERR_INVALID, "block size must divide the lattice");
    if (d->boundary == BBP_INFINITE && (d->bx % d->Lx || d->by % d->Ly))
        return fail(BBP_ERR_INVALID, "infinite block must be a multiple of the unit cell");
    if (d->dtype < 0 || d->dtype > 3) return fail(BBP_ERR_INVALID, "unknown dtype");
    if (d->prec < 0 || d->prec > 4) return fail(BBP_ERR_INVALID, "unknown precision");
    if (d->hermitian_basis != 0 && d->hermitian_basis != 1) return fail(BBP_ERR_INVALID, "hermitian_basis must be 0 or 1");
    if (d->fit_max_sweeps < 1 || d->fit_max_sweeps > 64) return fail(BBP_ERR_INVALID, "fit_max_sweeps must be 1..64");
    if (d->bx > 16 || d->by > 16) return fail(BBP_ERR_INVALID, "block sides are limited to 16 sites");
    if (d->Lx > 4096 || d->Ly > 4096) return fail(BBP_ERR_INVALID, "lattice sides are limited to 4096 sites");
    if (d->D > 16 || d->d > 64) return fail(BBP_ERR_INVALID, "D or d too large");
    if (d->init_mode != 0 && d->init_mode != 1) return fail(BBP_ERR_INVALID, "init_mode must be 0 or 1");
    if (d->warm_start < 0 || d->warm_start > 2) return fail(BBP_ERR_INVALID, "warm_start must be 0, 1 or 2");
    if (d->single_layer != 0 && d->single_layer != 1) return fail(BBP_ERR_INVALID, "single_layer must be 0 or 1");
    if (d->launch_mode != 0 && d->launch_mode != 1) return fail(BBP_ERR_INVALID, "launch_mode must be 0 or 1");
    if (d->keep_fp64 != 0 && d->keep_fp64 != 1) return fail(BBP_ERR_INVALID, "keep_fp64 must be 0 or 1");
    if (d->boundary == BBP_OBC ? (d->shift_x < 0 || d->shift_x >= d->bx || d->shift_y < 0 || d->shift_y >= d->by)
                               : (d->shift_x < 0 || d->shift_x >= d->Lx || d->shift_y < 0 || d->shift_y >= d->Ly))
        return fail(BBP_ERR_INVALID, "shifts: 0 <= shift < unit cell on infinite lattices, < block side with OBC");
    if (d->single_layer && (d->d != 1 || (d->dtype != BBP_F64 && d->dtype != BBP_F32)))
        return fail(BBP_ERR_INVALID, "a single-layer network has d = 1 and real tensors");
    return BBP_OK;
}

}  // extern "C"

// Geometry, layout and the whole sweep program, checked on the host; no device memory.
int bbp::plan_lattice(const bbp_lattice_desc* desc, bbp_lattice** out) {
    *out = nullptr;
    int rc = validate(desc);
    if (rc) return rc;
    bbp_lattice* L = new (std::nothrow) bbp_lattice();
    if (!L) return fail(BBP_ERR_OOM, "host allocation failed");
    L->desc = *desc;
    L->single = desc->single_layer != 0;
    L->K = L->single ? desc->D : desc->D * desc->D;
    // App. A's read-out bond 2 D^2 + 10 in terms of the network's leg dimension K
    if (L->desc.chi_exp <= 0) L->desc.chi_exp = std::max(desc->chi, 2 * L->K + 10);
    const bool in_cplx = desc->dtype == BBP_C128 || desc->dtype == BBP_C64;
    L->hb = in_cplx && (desc->prec != BBP_PREC_FP64 || desc->hermitian_basis != 0);
    L->cplx = in_cplx && !L->hb;
    L->ss = L->cplx ? 16 : 8;
    if (desc->boundary == BBP_OBC) {
        // block boundaries every bx columns from shift_x (every by rows from shift_y): with a
        // shift the blocks on the lattice edges are narrower (the shifted partition of the OBC
        // lattice, whose blocks straddling the periodic embedding's seam split into two)
        auto bounds = [](int L, int b, int sh) {
            std::vector<int> v{0};
            for (int x = sh; x < L; x += b)
                if (x > 0) v.push_back(x);
            v.push_back(L);
            return v;
        };
        L->xs = bounds(desc->Lx, desc->bx, desc->shift_x);
        L->ys = bounds(desc->Ly, desc->by, desc->shift_y);
    } else {
        L->xs = {0, desc->bx};
        L->ys = {0, desc->by};
    }
    L->nbx = (int)L->xs.size() - 1;
    L->nby = (int)L->ys.size() - 1;
    L->nblocks = L->nbx * L->nby;
    L->ntens = desc->Lx * desc->Ly;
    Program& pr = L->sweep;
    auto elem_alloc = [&](size_t elems) { return pr.arena_alloc(elems * (size_t)L->ss) / (size_t)L->ss; };
    L->one_off = elem_alloc(1);
    // tensors and double layers
    size_t raw_scalars = 0;
    for (int r = 0; r < (desc->boundary == BBP_OBC ? desc->Ly : desc->Ly); ++r)
        for (int c = 0; c < desc->Lx; ++c) {
            const auto dd = L->site_dims(r, c);
            L->tdims.push_back(dd);
            const size_t vol = (size_t)desc->d * dd[0] * dd[1] * dd[2] * dd[3];
            if (L->single) {
                // the network's own tensor is E: converted straight into its slot
                L->E_off.push_back(elem_alloc(vol));
                L->T_off.push_back(L->E_off.back());
            } else {
                L->T_off.push_back(elem_alloc(vol * (L->hb ? 2 : 1)));  // T stays complex in the Hermitian basis
                L->E_off.push_back(elem_alloc((size_t)dd[0] * dd[0] * dd[1] * dd[1] * dd[2] * dd[2] * dd[3] * dd[3]));
            }
            raw_scalars += vol;
        }
    L->T_elems = raw_scalars;
    const int in_ss = (desc->dtype == BBP_F64) ? 8 : (desc->dtype == BBP_C128) ? 16 : (desc->dtype == BBP_F32) ? 4 : 8;
    L->raw_bytes = raw_scalars * in_ss;
    L->raw_off = pr.arena_alloc(L->raw_bytes);
    // items and the message store
    L->item_of.assign(L->nblocks * 4, -1);
    for (int blk = 0; blk < L->nblocks; ++blk)
        for (int dir = 0; dir < 4; ++dir) {
            if (L->neighbour(blk, dir) < 0) continue;
            Item I;
            I.block = blk;
            I.dir = dir;
            I.msgid = 4 * blk + dir;
            int bh, bw;
            L->block_size(blk, bh, bw);
            I.b = (dir == DIR_LEFT || dir == DIR_RIGHT) ? bh : bw;
            std::vector<int> ph(I.b, L->K);
            I.mb = bond_caps(ph, desc->chi);
            L->item_of[blk * 4 + dir] = (int)L->items.size();
            L->items.push_back(I);
        }
    size_t off = 0;
    for (auto& I : L->items) {
        I.region_off = off;
        for (int s = 0; s < I.b; ++s) {
            I.site_off.push_back(off - I.region_off);
            off += (size_t)I.mb[s] * L->K * I.mb[s + 1];
            off = (off + 1) & ~(size_t)1;  // keep every site 16-byte aligned
        }
        I.region_elems = off - I.region_off;
    }
    L->msg_elems = std::max<size_t>(off, 2);
    L->msg_cur = elem_alloc(L->msg_elems);
    L->msg_new = elem_alloc(L->msg_elems);
    if (desc->prec != BBP_PREC_FP64) {
        L->mixed = true;
        MixCtx& cx = L->cx;
        cx.ss = L->ss;
        cx.tck = (desc->prec == BBP_PREC_BF16 || desc->prec == BBP_PREC_BF16X3) ? 1 : 0;
        cx.x3 = desc->prec == BBP_PREC_TF32X3 || desc->prec == BBP_PREC_BF16X3;
        cx.esz = cx.tck == 0 ? 4 : 2;
        cx.pe = 16 / cx.esz;
        cx.lpk = cx.tck == 0 ? 4 : 3;
        cx.tco = cx.tck == 0 ? 1 : 2;
        cx.qr_f32 = desc->keep_fp64 == 0;
        pr.tc_kind = cx.tck;
        // the constant 1 as a K = 1 operand row (16 bytes; a split one has a zero lo plane)
        L->one_lp = pr.lp_alloc(16 / cx.esz, cx.esz, cx.x3);
        L->one_lp_b = L->one_lp;
        const size_t errw = pr.arena_alloc(sizeof(int));
        L->d_tcerr = (int*)(uintptr_t)errw;
        for (int t = 0; t < L->ntens; ++t) {
            std::array<size_t, 4> el{}, er{};
            for (int dir = 0; dir < 4; ++dir) {
                const View4 o = L->E_view(t, dir);
                el[dir] = pr.lp_alloc((size_t)o.q * o.w2 * padded(cx, (long long)o.w * o.p), cx.esz, cx.x3);
                er[dir] = pr.lp_alloc((size_t)o.w * o.q * padded(cx, (long long)o.p * o.w2), cx.esz, cx.x3);
            }
            L->EL_off.push_back(el);
            L->ER_off.push_back(er);
        }
    }
    rc = plan_sweep(L);
    if (rc) {
        delete L;
        return rc;
    }
    {
        const std::string v = pr.validate();
        if (!v.empty()) {
            delete L;
            return fail(BBP_ERR_INVALID, "internal plan check: " + v);
        }
    }
    L->arena_bytes = pr.arena_used;
    *out = L;
    return BBP_OK;
}

extern "C" {

int bbp_lattice_footprint(const bbp_lattice_desc* desc, size_t* bytes) try {
    if (!bytes) return fail(BBP_ERR_INVALID, "bytes is NULL");
    bbp_lattice* L = nullptr;
    int rc = plan_lattice(desc, &L);
    if (rc) return rc;
    *bytes = planned_bytes(L);
    delete L;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_create_lattice(const bbp_lattice_desc* desc, bbp_lattice** out) try {
    if (!out) return fail(BBP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    bbp_lattice* L = nullptr;
    int rc = plan_lattice(desc, &L);
    if (rc) return rc;
    Program& pr = L->sweep;
    cudaError_t e = cudaSuccess;
    if (desc->stream == nullptr) {
        e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
        L->own_stream = e == cudaSuccess;
    } else {
        L->stream = (cudaStream_t)desc->stream;
    }
    // one arena for everything, stream-ordered so that creating a lattice never waits
    // for the kernels of another
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&L->arena, L->arena_bytes, L->stream);
    if (e != cudaSuccess) {
        L->arena = nullptr;
        bbp_destroy(L);
        return fail(BBP_ERR_OOM, std::string("arena of ") + std::to_string(L->arena_bytes) + " bytes: " + cudaGetErrorString(e));
    }
    char* base = L->arena;
    pr.relocate(base);
    pr.status = (int*)(base + (uintptr_t)L->d_status);
    L->d_status = pr.status;
    if (L->mixed) {
        L->d_tcerr = (int*)(base + (uintptr_t)L->d_tcerr);
        pr.tc_err = L->d_tcerr;
        cudaError_t em = pr.encode_maps(base);
        if (em != cudaSuccess) {
            bbp_destroy(L);
            return fail(BBP_ERR_CUDA, std::string("tensor map encoding: ") + cudaGetErrorString(em));
        }
    }
    L->d_resid_terms = (double*)(base + (uintptr_t)L->d_resid_terms);
    L->d_residual = (double*)(base + (uintptr_t)L->d_residual);
    L->d_sweep = (int*)(base + (uintptr_t)L->d_sweep);
    e = pr.upload_tasks(L->stream);
    if (e == cudaSuccess) {
        L->h_pinned = pinned_get();
        if (!L->h_pinned) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->arena, 0, L->arena_bytes, L->stream);
    if (e == cudaSuccess) {
        double one[2] = {1.0, 0.0};
        e = cudaMemcpyAsync(base + L->one_off * L->ss, one, L->ss, cudaMemcpyHostToDevice, L->stream);
    }
    if (e == cudaSuccess && L->mixed) {
        // the constant 1 as a K = 1 operand row; a split operand's lo plane stays zero (the
        // arena was cleared above)
        static const float one_f[4] = {1.0f, 0.0f, 0.0f, 0.0f};
        static const unsigned short one_b[8] = {0x3F80, 0, 0, 0, 0, 0, 0, 0};
        const bool bf = L->cx.tck == 1;
        e = cudaMemcpyAsync(base + L->one_lp, bf ? (const void*)one_b : (const void*)one_f, 16, cudaMemcpyHostToDevice,
                            L->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
        bbp_destroy(L);
        return fail(BBP_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = L;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

void bbp_destroy(bbp_lattice* L) try {
    if (!L) return;
    // waits for this lattice's own work only; the frees are stream-ordered
    if (L->stream) cudaStreamSynchronize(L->stream);
    L->sweep.free_all(L->stream);
    if (L->arena) cudaFreeAsync(L->arena, L->stream);
    if (L->stream) cudaStreamSynchronize(L->stream);
    if (L->h_pinned) pinned_put(L->h_pinned);
    if (L->done) cudaEventDestroy(L->done);
    if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
    delete L;
} catch (...) {
    abi_error();
}

// Initial messages (App. A: messages start from a chosen state; init_mode 0 is the
// product of delta_{ket,bra}, init_mode 1 a random positive MPDO of bond 1; on a
// single-layer network the all-ones product or positive uniform entries), each
// normalised to unit 2-norm with <I|m> (<1|m>) > 0: one task per message for k_msg_init.
static std::vector<MsgInitTask> init_tasks(bbp_lattice* L) {
    std::vector<MsgInitTask> ts;
    char* base = L->arena;
    for (int it = 0; it < (int)L->items.size(); ++it) {
        const Item& I = L->items[it];
        MsgInitTask t{};
        t.nsites = I.b;
        t.K = L->K;
        t.D = L->desc.D;
        t.mode = L->desc.init_mode;
        t.single = L->single ? 1 : 0;
        t.hb = L->hb ? 1 : 0;
        t.cw = L->cplx ? 2 : 1;
        t.seed = L->desc.seed;
        t.stream = stream_id(2, 0, (uint64_t)I.msgid, 0, 0);
        for (int s = 0; s < I.b; ++s) {
            // element [a=0][k][b=0] of a site with bonds (mb[s], mb[s+1]) sits at k * mb[s+1]
            t.dst[s] = (double*)(base + (L->msg_cur + I.region_off + I.site_off[s]) * L->ss);
            t.kstride[s] = I.mb[s + 1];
        }
        ts.push_back(t);
    }
    return ts;
}

int bbp_set_tensors(bbp_lattice* L, const void* data, int on_device) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (!data) return fail(BBP_ERR_INVALID, "data is NULL");
    char* base = L->arena;
    cudaStream_t st = L->stream;
    CKR(cudaMemcpyAsync(base + L->raw_off, data, L->raw_bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // convert into the compute type, tensor by tensor (raw is packed, T slabs are aligned)
    size_t in_scalar = 0;
    const int in_ss = (L->desc.dtype == BBP_F64) ? 8 : (L->desc.dtype == BBP_C128) ? 16 : (L->desc.dtype == BBP_F32) ? 4 : 8;
    std::vector<DLTask> dl;
    long long maxout = 1;
    for (int t = 0; t < L->ntens; ++t) {
        const auto& dd = L->tdims[t];
        const long long vol = (long long)L->desc.d * dd[0] * dd[1] * dd[2] * dd[3];
        CKR(launch_convert(base + L->raw_off + in_scalar * in_ss, L->desc.dtype, base + L->T_off[t] * L->ss, vol,
                           L->cplx || L->hb, st));
        in_scalar += vol;
        if (L->single) continue;  // E is the converted tensor itself
        DLTask k{};
        k.T = base + L->T_off[t] * L->ss;
        k.E = base + L->E_off[t] * L->ss;
        k.O = nullptr;
        k.d = L->desc.d;
        k.Du = dd[0]; k.Dl = dd[1]; k.Dd = dd[2]; k.Dr = dd[3];
        k.hb = L->hb ? 1 : 0;
        dl.push_back(k);
        maxout = std::max(maxout, (long long)dd[0] * dd[0] * dd[1] * dd[1] * dd[2] * dd[2] * dd[3] * dd[3]);
    }
    AsyncBuffer dlb(st);
    if (!dl.empty()) {
        CKR(cudaMallocAsync(&dlb.p, dl.size() * sizeof(DLTask), st));
        DLTask* d_dl = (DLTask*)dlb.p;
        CKR(cudaMemcpyAsync(d_dl, dl.data(), dl.size() * sizeof(DLTask), cudaMemcpyHostToDevice, st));
        if (L->hb)
            CKR(launch_double_layer_hb(d_dl, (int)dl.size(), maxout, st));
        else
            CKR(launch_double_layer(d_dl, (int)dl.size(), maxout, L->cplx, st));
    }
    if (L->mixed) {
        // low-precision operand layouts of every double-layer tensor in every frame
        std::vector<RelayoutTask> rt;
        long long mx = 1;
        const MixCtx& cx = L->cx;
        for (int t = 0; t < L->ntens; ++t)
            for (int dir = 0; dir < 4; ++dir) {
                const View4 o = L->E_view(t, dir);
                for (int order = 0; order < 2; ++order) {
                    RelayoutTask r{};
                    r.src = base + o.off * L->ss;
                    r.src_kind = 0;
                    r.dst_kind = cx.lpk;
                    if (order == 0) {
                        r.dst = base + L->EL_off[t][dir];  // OL[w2][q][pad(w p)]
                        const long long wp = padded(cx, (long long)o.w * o.p);
                        r.d[0] = o.w2; r.d[1] = o.q; r.d[2] = o.w; r.d[3] = o.p;
                        r.ss[0] = o.sw2; r.ss[1] = o.sq; r.ss[2] = o.sw; r.ss[3] = o.sp;
                        r.ds[0] = (long long)o.q * wp; r.ds[1] = wp; r.ds[2] = o.p; r.ds[3] = 1;
                        r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? L->sweep.plane_of(L->EL_off[t][dir]) : 0;
                    } else {
                        r.dst = base + L->ER_off[t][dir];
                        const long long pw = padded(cx, (long long)o.p * o.w2);
                        r.d[0] = o.w; r.d[1] = o.q; r.d[2] = o.p; r.d[3] = o.w2;
                        r.ss[0] = o.sw; r.ss[1] = o.sq; r.ss[2] = o.sp; r.ss[3] = o.sw2;
                        r.ds[0] = (long long)o.q * pw; r.ds[1] = pw; r.ds[2] = o.w2; r.ds[3] = 1;
                        r.x3 = cx.x3 ? 1 : 0; r.kseg = cx.x3 ? L->sweep.plane_of(L->ER_off[t][dir]) : 0;
                    }
                    mx = std::max(mx, (long long)o.w * o.p * o.q * o.w2);
                    rt.push_back(r);
                }
            }
        AsyncBuffer rtb(st);
        CKR(cudaMallocAsync(&rtb.p, rt.size() * sizeof(RelayoutTask), st));
        RelayoutTask* d_rt = (RelayoutTask*)rtb.p;
        CKR(cudaMemcpyAsync(d_rt, rt.data(), rt.size() * sizeof(RelayoutTask), cudaMemcpyHostToDevice, st));
        CKR(launch_relayout(d_rt, (int)rt.size(), mx, st));
        CKR(cudaMemsetAsync(L->d_tcerr, 0, sizeof(int), st));
    }
    // initial messages, built on the device into the zeroed message region
    CKR(cudaMemsetAsync(base + L->msg_cur * L->ss, 0, L->msg_elems * L->ss, st));
    {
        const std::vector<MsgInitTask> mt = init_tasks(L);
        if (!mt.empty()) {
            AsyncBuffer mb(st);
            CKR(cudaMallocAsync(&mb.p, mt.size() * sizeof(MsgInitTask), st));
            CKR(cudaMemcpyAsync(mb.p, mt.data(), mt.size() * sizeof(MsgInitTask), cudaMemcpyHostToDevice, st));
            CKR(launch_msg_init((const MsgInitTask*)mb.p, (int)mt.size(), st));
        }
    }
    CKR(cudaMemsetAsync(L->d_sweep, 0, sizeof(int), st));
    CKR(cudaMemsetAsync(L->d_status, 0, sizeof(int), st));
    CKR(cudaStreamSynchronize(st));
    L->has_tensors = true;
    L->sweeps = 0;
    L->first_residual = L->last_residual = 0;
    CKR(L->sweep.reset_loop_totals(st));  // a new solve restarts the loop statistics
    return BBP_OK;
} catch (...) {
    return abi_error();
}

static int ensure_graph(bbp_lattice* L) {
    Program& pr = L->sweep;
    if (pr.exec) return BBP_OK;
    CKR(pr.build_graph(L->stream, L->d_sweep, L->desc.seed));
    return BBP_OK;
}

}  // extern "C"

namespace bbp {

// Queue one sweep (graph launch) and the copies of its residual and error words into
// pinned memory, then record the sweep's event.  Asynchronous.
int sweep_launch(bbp_lattice* L) {
    if (L->desc.launch_mode == 1) {
        // the sweep's kernels one by one; every fit loop runs its maximum count, the fits that
        // have met the stop rule skipping their work (the graph's result, launch by launch)
        if (!L->direct_ready) {
            CKR(L->sweep.init_loops(L->stream, false, nullptr));
            L->direct_ready = true;
        }
        CKR(L->sweep.launch_all(L->stream, L->d_sweep, L->desc.seed));
    } else {
        int rc = ensure_graph(L);
        if (rc) return rc;
        CKR(cudaGraphLaunch(L->sweep.exec, L->stream));
    }
    CKR(cudaMemcpyAsync(&L->h_pinned->residual, L->d_residual, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CKR(cudaMemcpyAsync(&L->h_pinned->status, L->d_status, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
    if (L->mixed) CKR(cudaMemcpyAsync(&L->h_pinned->tc_err, L->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
    CKR(cudaEventRecord(L->done, L->stream));
    return BBP_OK;
}

bool sweep_ready(bbp_lattice* L) { return cudaEventQuery(L->done) != cudaErrorNotReady; }

size_t planned_bytes(const bbp_lattice* L) {
    return L->arena_bytes + L->sweep.tcs.size() * sizeof(TCTask) + L->sweep.gc.size() * sizeof(GTask) +
           L->sweep.qr.size() * sizeof(QRTask);
}

// After the sweep's event: account for it and apply the stop rule.  *stop is set when
// the residual meets the tolerance (absolute, or relative to the first sweep).
int sweep_collect(bbp_lattice* L, double* residual, bool* stop) {
    CKR(cudaEventSynchronize(L->done));
    L->sweeps++;
    const double r = L->h_pinned->residual;
    if (residual) *residual = r;
    if (L->mixed && L->h_pinned->tc_err) return fail(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its bound");
    if (L->h_pinned->status != 0 || !std::isfinite(r))
        return fail(BBP_ERR_NUMERIC, "a message or column MPS has zero or non-finite norm");
    if (L->sweeps == 1) L->first_residual = r;
    L->last_residual = r;
    const double crit = L->desc.stop_relative ? (L->first_residual > 0 ? r / L->first_residual : 0.0) : r;
    if (stop) *stop = crit < L->desc.tol;
    return BBP_OK;
}

}  // namespace bbp

extern "C" {

int bbp_sweep(bbp_lattice* L, int n_sweeps, double* residual_out, int* sweeps_done) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (!L->has_tensors) return fail(BBP_ERR_STATE, "bbp_set_tensors has not been called");
    const bool fixed = n_sweeps > 0;
    const int cap = fixed ? n_sweeps : std::max(1, L->desc.max_sweeps);
    int done = 0;
    double r = 0.0;
    bool converged = fixed;
    if (L->items.empty()) {  // a single block without neighbours: nothing to iterate
        if (residual_out) *residual_out = 0.0;
        if (sweeps_done) *sweeps_done = 0;
        return BBP_OK;
    }
    for (int k = 0; k < cap; ++k) {
        int rc = sweep_launch(L);
        bool stop = false;
        if (!rc) rc = sweep_collect(L, &r, &stop);
        done += rc ? 0 : 1;
        if (rc) {
            if (residual_out) *residual_out = r;
            if (sweeps_done) *sweeps_done = done;
            return rc;
        }
        if (!fixed && stop) {
            converged = true;
            break;
        }
    }
    if (residual_out) *residual_out = r;
    if (sweeps_done) *sweeps_done = done;
    return converged ? BBP_OK : BBP_NOT_CONVERGED;
} catch (...) {
    return abi_error();
}

int bbp_get_message(bbp_lattice* L, int block, int dir, int* nsites, int* bonds, double* out) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (block < 0 || block >= L->nblocks || dir < 0 || dir > 3 || L->item_of[block * 4 + dir] < 0)
        return fail(BBP_ERR_INVALID, "no such message");
    const int it = L->item_of[block * 4 + dir];
    const Item& I = L->items[it];
    if (nsites) *nsites = I.b;
    if (bonds)
        for (int s = 0; s <= I.b; ++s) bonds[s] = I.mb[s];
    if (out) {
        size_t o = 0;
        for (int s = 0; s < I.b; ++s) {
            const View3 v = L->msg_site(it, s, true);
            const size_t cnt = (size_t)v.a * v.k * v.b * (L->cplx ? 2 : 1);
            CKR(cudaMemcpyAsync(out + o, L->arena + v.off * L->ss, cnt * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
            o += cnt;
        }
        CKR(cudaStreamSynchronize(L->stream));
    }
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_set_message(bbp_lattice* L, int block, int dir, const double* in) try {
    if (!L || !in) return fail(BBP_ERR_INVALID, "NULL argument");
    if (block < 0 || block >= L->nblocks || dir < 0 || dir > 3 || L->item_of[block * 4 + dir] < 0)
        return fail(BBP_ERR_INVALID, "no such message");
    const int it = L->item_of[block * 4 + dir];
    const Item& I = L->items[it];
    size_t o = 0;
    for (int s = 0; s < I.b; ++s) {
        const View3 v = L->msg_site(it, s, true);
        const size_t cnt = (size_t)v.a * v.k * v.b * (L->cplx ? 2 : 1);
        CKR(cudaMemcpyAsync(L->arena + v.off * L->ss, in + o, cnt * sizeof(double), cudaMemcpyHostToDevice, L->stream));
        o += cnt;
    }
    CKR(cudaStreamSynchronize(L->stream));
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_time_kernels(bbp_lattice* L, int cls, int reps, double* ms, long long* launches, double* flops, double* bytes) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (!L->has_tensors) return fail(BBP_ERR_STATE, "bbp_set_tensors has not been called");
    if (cls < 0 || cls > 2 || reps < 1) return fail(BBP_ERR_INVALID, "kernel class must be 0..2 and reps >= 1");
    EventPair ev;
    CKR(cudaEventCreate(&ev.a));
    CKR(cudaEventCreate(&ev.b));
    cudaEvent_t a = ev.a, b = ev.b;
    long long n = 0;
    double f = 0, by = 0;
    CKR(L->sweep.reset_active(L->stream));
    CKR(cudaEventRecord(a, L->stream));
    for (int r = 0; r < reps; ++r) CKR(L->sweep.launch_class(L->stream, L->d_sweep, L->desc.seed, cls, &n, &f, &by));
    CKR(cudaEventRecord(b, L->stream));
    CKR(cudaEventSynchronize(b));
    float t = 0;
    CKR(cudaEventElapsedTime(&t, a, b));
    if (L->mixed) {
        int te = 0;
        CKR(cudaMemcpy(&te, L->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost));
        if (te) return fail(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its bound");
    }
    if (ms) *ms = t / reps;
    if (launches) *launches = n;
    if (flops) *flops = f;
    if (bytes) *bytes = by;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

// Time `reps` launches of step si (after one warm-up) with CUDA events on the handle's stream.
static cudaError_t time_step(bbp_lattice* L, size_t si, int reps, cudaEvent_t a, cudaEvent_t b, float* ms) {
    Program& pr = L->sweep;
    cudaStream_t st = L->stream;
    cudaError_t e = pr.launch_step(pr.steps[si], st, L->d_sweep, L->desc.seed);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = pr.launch_step(pr.steps[si], st, L->d_sweep, L->desc.seed);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    return e;
}

int bbp_time_steps(bbp_lattice* L, int reps, int cap, bbp_step_time* out, int* n_steps) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (reps < 1 || cap < 0 || (cap > 0 && !out) || !n_steps) return fail(BBP_ERR_INVALID, "bad arguments");
    if (!L->has_tensors) return fail(BBP_ERR_STATE, "bbp_set_tensors has not been called");
    Program& pr = L->sweep;
    EventPair ev;
    CKR(cudaEventCreate(&ev.a));
    CKR(cudaEventCreate(&ev.b));
    CKR(pr.reset_active(L->stream));
    int n = 0;
    for (size_t si = 0; si < pr.steps.size(); ++si) {
        const Step& s = pr.steps[si];
        const int cls = pr.step_class_of(s);
        if (cls > 2) continue;
        if (n < cap) {
            bbp_step_time& r = out[n];
            r = bbp_step_time{};
            r.index = (int)si;
            r.kernel_class = cls;
            r.tasks = s.count;
            r.tile_n = s.kind == ST_TC ? s.aux : 0;
            pr.step_work(s, &r.flops, &r.bytes, &r.max_m, &r.max_n, &r.max_k);
            float t = 0.0f;
            CKR(time_step(L, si, reps, ev.a, ev.b, &t));
            r.ms = t / reps;
        }
        ++n;
    }
    *n_steps = n;
    if (L->mixed) {
        int te = 0;
        CKR(cudaMemcpy(&te, L->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost));
        if (te) return fail(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its bound");
    }
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_autotune(bbp_lattice* L, int reps, double* ms_before, double* ms_after, int* steps_changed) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (reps < 1) return fail(BBP_ERR_INVALID, "reps must be >= 1");
    if (!L->has_tensors) return fail(BBP_ERR_STATE, "bbp_set_tensors has not been called");
    if (L->sweeps > 0 || L->sweep.exec) return fail(BBP_ERR_STATE, "autotune must run before the first sweep");
    double before = 0.0, after = 0.0;
    int changed = 0;
    Program& pr = L->sweep;
    cudaStream_t st = L->stream;
    EventPair ev;
    CKR(cudaEventCreate(&ev.a));
    CKR(cudaEventCreate(&ev.b));
    cudaEvent_t a = ev.a, b = ev.b;
    CKR(pr.reset_active(st));  // every fit stage runs, as in a first sweep
    const int ek = L->cx.tck == 0 ? 32 : 64;  // K elements per k-block
    for (size_t si = 0; si < pr.steps.size(); ++si) {
        const Step s0 = pr.steps[si];
        if (s0.kind == ST_TC && L->mixed) {
            // tensor-core tiles: width BN and TMA ring depth
            int nmax = 1, kmax = 1;
            for (int i = 0; i < s0.count; ++i) {
                nmax = std::max(nmax, pr.tcs[s0.first + i].N);
                kmax = std::max(kmax, (pr.tcs[s0.first + i].K + ek - 1) / ek * (pr.tcs[s0.first + i].nseg == 3 ? 3 : 1));
            }
            const int bn0 = s0.aux, d0 = (s0.aux2 >> 8) & 0xFF, k0 = std::max(1, (s0.aux2 >> 16) & 0xFF);
            int best_bn = bn0, best_d = d0, best_k = k0;
            float best = -1.0f, t0 = -1.0f;
            for (int bn : {32, 64, 128, 256}) {
                if (bn > 32 && bn / 2 >= nmax) break;  // wider tiles than the widest result
                for (int ksub : {1, 2}) {                 // k-blocks per ring stage
                    const int need = (kmax + ksub - 1) / ksub;  // stages the K extent fills
                    if (ksub > 1 && kmax < 2) break;
                    for (int depth : {2, 3, 4, 6, 8}) {
                        if (depth > std::max(2, need) || depth > tc_max_stages(bn, ksub)) break;
                        CKR(pr.tc_retile(si, bn, depth, L->arena, (size_t)-1, nullptr, st, ksub));
                        float t = 0.0f;
                        CKR(time_step(L, si, reps, a, b, &t));
                        if (bn == bn0 && depth == d0 && ksub == k0) t0 = t;
                        if (best < 0.0f || t < best) {
                            best = t;
                            best_bn = bn;
                            best_d = depth;
                            best_k = ksub;
                        }
                    }
                }
            }
            CKR(pr.tc_retile(si, best_bn, best_d, L->arena, (size_t)-1, nullptr, st, best_k));
            if (best_bn != bn0 || best_d != d0 || best_k != k0) ++changed;
            before += (t0 >= 0.0f ? t0 : best) / reps;
            after += best / reps;
        } else if (s0.kind == ST_QR && !(s0.aux2 & QR_F32) && qr_cluster_fits(s0.aux, s0.n, pr.cplx, 1)) {
            // QR/LQ: cluster size (0: the built-in rule); the result is the same for every C
            int best_c = 0;
            float best = -1.0f, t0 = -1.0f;
            for (int c = 0; c <= 8; ++c) {
                if (c > 0 && !qr_cluster_fits(s0.aux, s0.n, pr.cplx, c)) continue;
                pr.steps[si].aux2 = c;
                float t = 0.0f;
                CKR(time_step(L, si, reps, a, b, &t));
                if (c == 0) t0 = t;
                if (best < 0.0f || t < best * 0.98f) {  // keep the rule unless a size is clearly faster
                    best = t;
                    best_c = c;
                }
            }
            pr.steps[si].aux2 = best_c;
            if (best_c != 0) ++changed;
            before += t0 / reps;
            after += best / reps;
        }
    }
    CKR(pr.reset_loop_totals(st));  // the timings ran no fit of the solve: statistics restart
    CKR(cudaStreamSynchronize(st));
    int te = 0;
    if (L->mixed) CKR(cudaMemcpy(&te, L->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (te) return fail(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its bound");
    if (ms_before) *ms_before = before;
    if (ms_after) *ms_after = after;
    if (steps_changed) *steps_changed = changed;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_get_stats(bbp_lattice* L, bbp_stats* out) try {
    if (!L || !out) return fail(BBP_ERR_INVALID, "NULL argument");
    memset(out, 0, sizeof(*out));
    const Program& pr = L->sweep;
    long long fs = 0, fits = 0;
    std::vector<const int*> seen;
    for (const auto& t : pr.chk) {
        if (std::find(seen.begin(), seen.end(), t.counter) != seen.end()) continue;
        seen.push_back(t.counter);
        int v = 0;
        CKR(cudaMemcpy(&v, t.counter, sizeof(int), cudaMemcpyDeviceToHost));
        fs += v;
        fits++;
    }
    long long launches = 0;
    double fl = 0, qfl = 0;
    long long iters = 0;
    if (L->sweeps > 0) CKR(pr.executed(L->sweeps, &launches, &fl, &qfl, &iters));
    out->fit_loop_iters = iters;
    out->fit_sweeps = fs;
    out->fits = fits * (long long)L->sweeps;
    out->flops = fl + L->readout_flops;
    out->qr_flops = qfl;
    out->kernels = launches + L->readout_kernels;
    out->sweeps = L->sweeps;
    out->last_residual = L->last_residual;
    out->first_residual = L->first_residual;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

}  // extern "C"
