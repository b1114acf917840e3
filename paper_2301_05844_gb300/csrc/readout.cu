// bbp_expect: expectation values from a block and its converged incoming messages.
//
// App. A: once the messages have converged, the block plus its four incoming
// messages is contracted by bMPS with the larger bond chi = 2D^2+10 (Fig. 1(f)).
// Here every region (a block, or two neighbouring blocks merged for a pair that
// crosses a block edge) gets its left and right environment columns L_c, R_c from
// the same lockstep zip-up fits as the sweep, and each term is the exact
// top-to-bottom closing L_c . column(s) . R_c with E^O at the operator sites;
// <O> = N_O / N_I is formed in FP64.  The closings of one column strip share its top
// and bottom environments, so a term costs the rows that carry its operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <complex>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "bbp.h"
#include "bbp_internal.h"
#include "engine.h"
#include "lattice.h"

using namespace bbp;

namespace {

struct Op4 {
    size_t off = 0;
    int u = 1, l = 1, d = 1, r = 1;
    long long su = 0, sl = 0, sd = 0, sr = 0;
};

struct Region {
    int rid = 0, r0 = 0, c0 = 0, h = 0, w = 0;
    std::vector<int> blocks;
    std::vector<View3> in[4];
    int sweepL = -1, sweepR = -1;  // indices into the column-sweep list
};

struct Closing {
    int region = 0, col = 0, ncols = 1;
    std::vector<std::pair<int, int>> pos;     // local (row, col) of the operator sites
    std::vector<std::vector<double>> ops;     // d*d scalars each (S layout); impurity tensors
                                              // on a single-layer network
};

Op4 op_from_top(const View3& t) {
    Op4 o;
    o.off = t.off; o.u = 1; o.l = t.a; o.d = t.k; o.r = t.b;
    o.su = 0; o.sl = t.sa; o.sd = t.sk; o.sr = t.sb;
    return o;
}
Op4 op_from_bottom(const View3& b) {
    Op4 o;
    o.off = b.off; o.u = b.k; o.l = b.a; o.d = 1; o.r = b.b;
    o.su = b.sk; o.sl = b.sa; o.sd = 0; o.sr = b.sb;
    return o;
}
Op4 op_contig(size_t off, int u, int l, int d, int r) {
    Op4 o;
    o.off = off; o.u = u; o.l = l; o.d = d; o.r = r;
    o.su = (long long)l * d * r; o.sl = (long long)d * r; o.sd = r; o.sr = 1;
    return o;
}

}  // namespace

#define CKR(expr)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) return fail(BBP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" int bbp_expect(bbp_lattice* L, const bbp_term* terms, int n_terms, double* out_re, double* out_im) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (!L->has_tensors) return fail(BBP_ERR_STATE, "bbp_set_tensors has not been called");
    if (n_terms < 0 || (n_terms > 0 && (!terms || !out_re))) return fail(BBP_ERR_INVALID, "bad term arguments");
    if (n_terms == 0) return BBP_OK;
    const bbp_lattice_desc& ds = L->desc;
    const int d = ds.d, ss = L->ss;
    const bool obc = ds.boundary == BBP_OBC;
    const int Wlat = obc ? ds.Lx : ds.bx, Hlat = obc ? ds.Ly : ds.by;

    // ---- regions and closings
    std::vector<Region> regions;
    std::map<int, int> region_of;
    auto get_region = [&](const std::vector<std::pair<int, int>>& rc, int& out) -> int {
        int rid, r0, c0, h, w;
        bool horiz = false;
        std::vector<int> blks;
        if (!obc) {
            rid = 0; r0 = 0; c0 = 0; h = ds.by; w = ds.bx;
            blks = {0};
        } else {
            for (auto& p : rc) blks.push_back(L->block_of(p.first, p.second));
            if (blks.size() == 1 || blks[0] == blks[1]) {
                rid = blks[0];
                L->block_origin(rid, r0, c0);
                L->block_size(rid, h, w);
                blks = {rid};
            } else {
                const int dr = std::abs(rc[0].first - rc[1].first), dc = std::abs(rc[0].second - rc[1].second);
                if (dr + dc != 1) return fail(BBP_ERR_INVALID, "a two-site term across blocks must be a nearest-neighbour pair");
                const int a = std::min(blks[0], blks[1]), b = std::max(blks[0], blks[1]);
                int ha, wa, hb, wb;
                L->block_origin(a, r0, c0);
                L->block_size(a, ha, wa);
                L->block_size(b, hb, wb);
                horiz = dc == 1;
                if (horiz) {
                    rid = L->nblocks + 2 * a; h = ha; w = wa + wb;
                } else {
                    rid = L->nblocks + 2 * a + 1; h = ha + hb; w = wa;
                }
                blks = {a, b};
            }
        }
        auto it = region_of.find(rid);
        if (it != region_of.end()) {
            out = it->second;
            return BBP_OK;
        }
        Region R;
        R.rid = rid; R.r0 = r0; R.c0 = c0; R.h = h; R.w = w; R.blocks = blks;
        if (blks.size() == 1) {
            for (int dd = 0; dd < 4; ++dd) R.in[dd] = L->incoming(blks[0], dd);
        } else {
            std::vector<View3> ia[4], ib[4];
            for (int dd = 0; dd < 4; ++dd) {
                ia[dd] = L->incoming(blks[0], dd);
                ib[dd] = L->incoming(blks[1], dd);
            }
            auto cat = [](std::vector<View3> x, const std::vector<View3>& y) {
                x.insert(x.end(), y.begin(), y.end());
                return x;
            };
            if (horiz) {
                R.in[DIR_LEFT] = ia[DIR_LEFT]; R.in[DIR_RIGHT] = ib[DIR_RIGHT];
                R.in[DIR_UP] = cat(ia[DIR_UP], ib[DIR_UP]); R.in[DIR_DOWN] = cat(ia[DIR_DOWN], ib[DIR_DOWN]);
            } else {
                R.in[DIR_UP] = ia[DIR_UP]; R.in[DIR_DOWN] = ib[DIR_DOWN];
                R.in[DIR_LEFT] = cat(ia[DIR_LEFT], ib[DIR_LEFT]); R.in[DIR_RIGHT] = cat(ia[DIR_RIGHT], ib[DIR_RIGHT]);
            }
        }
        region_of[rid] = (int)regions.size();
        out = (int)regions.size();
        regions.push_back(R);
        return BBP_OK;
    };

    std::vector<Closing> closings;
    std::map<std::tuple<int, int, int>, int> norm_closing;
    struct TermPlan {
        std::vector<std::pair<int, std::complex<double>>> parts;  // (closing, coefficient)
        int denom = 0;
    };
    std::vector<TermPlan> tplan(n_terms);
    for (int t = 0; t < n_terms; ++t) {
        const bbp_term& T = terms[t];
        if (T.nsite < 1 || T.nsite > 2) return fail(BBP_ERR_INVALID, "term must have 1 or 2 sites");
        std::vector<std::pair<int, int>> rc;
        for (int k = 0; k < T.nsite; ++k) {
            if (!T.op_re[k]) return fail(BBP_ERR_INVALID, "operator is NULL");
            const int s = T.site[k];
            if (s < 0 || s >= Wlat * Hlat) return fail(BBP_ERR_INVALID, "site out of range");
            rc.push_back({s / Wlat, s % Wlat});
        }
        if (T.nsite == 2 && T.site[0] == T.site[1]) return fail(BBP_ERR_INVALID, "two-site term on one site");
        int ri;
        int rc_ = get_region(rc, ri);
        if (rc_) return rc_;
        const Region& R = regions[ri];
        std::vector<std::pair<int, int>> loc;
        int cmin = 1 << 30, cmax = -1;
        for (auto& p : rc) {
            loc.push_back({p.first - R.r0, p.second - R.c0});
            cmin = std::min(cmin, p.second - R.c0);
            cmax = std::max(cmax, p.second - R.c0);
        }
        if (cmax - cmin > 1) return fail(BBP_ERR_INVALID, "a two-site term must lie in one column or two adjacent columns");
        const int ncols = cmax - cmin + 1;
        // operator parts: complex lattices take the complex operator; real lattices
        // split O = O_re + i O_im into real closings with complex coefficients
        std::vector<std::vector<std::pair<std::vector<double>, std::complex<double>>>> parts(T.nsite);
        for (int k = 0; k < T.nsite; ++k) {
            // d x d operator, or the impurity tensor of the site on a single-layer network
            size_t nop = (size_t)d * d;
            if (L->single) {
                const auto dd = L->site_dims(rc[k].first, rc[k].second);
                nop = (size_t)dd[0] * dd[1] * dd[2] * dd[3];
            }
            std::vector<double> re(T.op_re[k], T.op_re[k] + nop), im(nop, 0.0);
            if (T.op_im[k]) im.assign(T.op_im[k], T.op_im[k] + nop);
            if (L->cplx) {
                std::vector<double> z(2 * d * d);
                for (int j = 0; j < d * d; ++j) {
                    z[2 * j] = re[j];
                    z[2 * j + 1] = im[j];
                }
                parts[k].push_back({z, 1.0});
            } else if (L->hb) {
                // Hermitian basis: O = H + i A with H = (O + O^dagger)/2 and
                // A = (O - O^dagger)/(2i) both Hermitian, so that each E^H, E^A is real there;
                // uploaded as complex d x d matrices for the double-layer kernel
                std::vector<double> h(2 * d * d), a(2 * d * d);
                bool has_h = false, has_a = false;
                for (int r = 0; r < d; ++r)
                    for (int c = 0; c < d; ++c) {
                        const int j = r * d + c, jt = c * d + r;
                        const double zr = re[j] - re[jt], zi = im[j] + im[jt];  // O_rc - conj(O_cr)
                        h[2 * j] = 0.5 * (re[j] + re[jt]);
                        h[2 * j + 1] = 0.5 * (im[j] - im[jt]);
                        a[2 * j] = 0.5 * zi;
                        a[2 * j + 1] = -0.5 * zr;
                        has_h |= h[2 * j] != 0.0 || h[2 * j + 1] != 0.0;
                        has_a |= a[2 * j] != 0.0 || a[2 * j + 1] != 0.0;
                    }
                if (has_h || !has_a) parts[k].push_back({h, 1.0});
                if (has_a) parts[k].push_back({a, std::complex<double>(0.0, 1.0)});
            } else {
                bool has_re = false, has_im = false;
                for (size_t j = 0; j < nop; ++j) {
                    has_re |= re[j] != 0.0;
                    has_im |= im[j] != 0.0;
                }
                if (has_re || !has_im) parts[k].push_back({re, 1.0});
                if (has_im) parts[k].push_back({im, std::complex<double>(0.0, 1.0)});
            }
        }
        auto add_closing = [&](const std::vector<std::vector<double>>& ops, std::complex<double> coef) {
            Closing C;
            C.region = ri; C.col = cmin; C.ncols = ncols;
            C.pos = loc;
            C.ops = ops;
            tplan[t].parts.push_back({(int)closings.size(), coef});
            closings.push_back(C);
        };
        if (T.nsite == 1) {
            for (auto& a : parts[0]) add_closing({a.first}, a.second);
        } else {
            for (auto& a : parts[0])
                for (auto& b : parts[1]) add_closing({a.first, b.first}, a.second * b.second);
        }
        const auto key = std::make_tuple(ri, cmin, ncols);
        auto nc = norm_closing.find(key);
        if (nc == norm_closing.end()) {
            Closing C;
            C.region = ri; C.col = cmin; C.ncols = ncols;
            norm_closing[key] = (int)closings.size();
            tplan[t].denom = (int)closings.size();
            closings.push_back(C);
        } else {
            tplan[t].denom = nc->second;
        }
    }

    // ---- the read-out program: env columns (fits with chi_exp), then closings
    Program pr;
    pr.cplx = L->cplx;
    const size_t split = (L->arena_bytes + 255) & ~(size_t)255;
    pr.arena_used = split;
    pr.parent = &L->sweep;  // buffers below `split` are the lattice's
    pr.split = split;
    pr.warm_ctr_off = L->sweep.warm_ctr_off;
    auto elem_alloc = [&](size_t elems) { return pr.arena_alloc(elems * (size_t)ss) / (size_t)ss; };
    std::vector<ColumnSweep> cs;
    for (auto& R : regions) {
        for (int side = 0; side < 2; ++side) {
            ColumnSweep s;
            s.dir = side == 0 ? DIR_LEFT : DIR_RIGHT;
            s.r0 = R.r0; s.c0 = R.c0; s.bh = R.h; s.bw = R.w;
            s.fm = L->frame_msgs(s.dir, R.in);
            s.chi = ds.chi_exp;
            s.keep = true;
            s.tag = 1;
            s.outer = (uint64_t)R.rid;
            s.msg = (uint64_t)side;
            // Warm read-out (desc->warm_start = 2, chi_exp = chi): a one-block region's
            // environment columns in this frame are the fits the sweep runs for the block's
            // message in the same direction; they start from that sweep's last fitted MPS of
            // each column.
            if (ds.warm_start == 2 && ds.chi_exp == ds.chi && R.blocks.size() == 1)
                for (const auto& I : L->items)
                    if (I.block == R.blocks[0] && I.dir == s.dir) s.warm_from = &I.fits;
            (side == 0 ? R.sweepL : R.sweepR) = (int)cs.size();
            cs.push_back(s);
        }
    }
    // The environment columns are fits like those of a sweep.  On a split-precision lattice
    // (TF32X3, BF16X3) they run on its tensor-core path (split contractions, FP64 QR, the same
    // fit tolerance); plain TF32 / BF16 lattices keep FP64 fits here, so that the read-out adds
    // no error of its own at their precision.  The closings and N_O / N_I are FP64 in every case.
    const bool tc_env = L->mixed && L->cx.x3;
    if (tc_env) {
        pr.tc_kind = L->cx.tck;
        pr.tc_err = L->d_tcerr;
    }
    int rc = plan_column_sweeps(L, pr, cs, ds.fit_max_sweeps, tc_env ? std::max(ds.fit_tol, fit_tol_floor(ds.prec)) : ds.fit_tol,
                                false, tc_env);
    if (rc) return rc;

    auto env_site = [&](const Region& R, bool left_env, int c, int i) -> View3 {
        // R env of column c: right edge absorbed down to c+1; L env: left edge up to c-1
        const ColumnSweep& s = cs[left_env ? R.sweepR : R.sweepL];
        const int W = R.w;
        int k = left_env ? (W - c) : (c + 1);  // frame column index of the kept fit
        if (k >= W) {  // the unabsorbed edge: [1, message, 1]
            if (i == 0 || i == R.h + 1) {
                View3 v;
                v.off = L->one_off;
                return v;
            }
            return s.fm.R[i - 1];
        }
        const FitSpec& f = s.fits[k];
        return contiguous3(f.Y[i], f.ybond[i], f.O[i].q, f.ybond[i + 1]);
    };

    // ---- closings, shared per column strip
    // A strip is one (region, first column, columns) group of closings.  Its top environments
    // T_i (rows 0..i-1 contracted; open legs: left env bond a, the strip's vertical leg(s) w,
    // right env bond b, stored [a][w][b]) and bottom environments G_i (rows i..h+1, the same
    // legs) are formed once; a closing with operators on rows i0..i1 contracts T_i0, those rows
    // with E^O at its operator sites, and G_(i1+1) (an inner product), and the strip's
    // N_I = <T_(h+1), G_(h+1)>.  These are the sums of the top-to-bottom closing L_c . column(s)
    // . R_c, in another order.
    struct Strip {
        int region = 0, col = 0, ncols = 1, norm = -1;
        std::vector<int> clos;
        std::vector<size_t> T, G;    // element offsets of T_i (i = 1..h+1) and G_i (i = 2..h+1)
        std::vector<size_t> eT, eG;  // byte offsets of their power-of-two exponents (FP32 closings)
        size_t chain = 0;            // their scalars
    };
    std::vector<Strip> strips;
    {
        std::map<std::tuple<int, int, int>, int> sid;
        for (size_t ci = 0; ci < closings.size(); ++ci) {
            const Closing& C = closings[ci];
            const auto key = std::make_tuple(C.region, C.col, C.ncols);
            auto it = sid.find(key);
            int k = 0;
            if (it == sid.end()) {
                k = (int)strips.size();
                sid[key] = k;
                Strip S;
                S.region = C.region; S.col = C.col; S.ncols = C.ncols;
                strips.push_back(S);
            } else {
                k = it->second;
            }
            if (C.pos.empty())
                strips[k].norm = (int)ci;
            else
                strips[k].clos.push_back((int)ci);
        }
    }
    const int K4max = L->K * L->K * L->K * L->K;
    const size_t nclos = closings.size();
    const size_t results = elem_alloc(nclos);
    // the ratios N_O / N_I, formed on the device: task descriptors, (re, im) per term, status
    static_assert(sizeof(RatioTask) % sizeof(double) == 0, "ratio tasks are uploaded as doubles");
    const size_t ratio_tasks = pr.arena_alloc((size_t)n_terms * sizeof(RatioTask));
    const size_t ratio_out = pr.arena_alloc((size_t)n_terms * 2 * sizeof(double));
    const size_t ratio_status = pr.arena_alloc(sizeof(int));
    auto row_op = [&](const Region& R, int c, int i, size_t eo_off, bool use_eo) -> Op4 {
        if (i == 0) return op_from_top(R.in[DIR_UP][c]);
        if (i == R.h + 1) return op_from_bottom(R.in[DIR_DOWN][c]);
        const int r = R.r0 + i - 1, cc = R.c0 + c;
        const auto dd = L->site_dims(r, cc);
        const size_t off = use_eo ? eo_off : L->E_off[L->tensor_index(r, cc)];
        if (L->single) return op_contig(off, dd[0], dd[1], dd[2], dd[3]);
        return op_contig(off, dd[0] * dd[0], dd[1] * dd[1], dd[2] * dd[2], dd[3] * dd[3]);
    };
    // leg dimensions of strip row i: (u, l, d, r) of its (fused) operator
    auto row_dims = [&](const Strip& S, int i) -> std::array<long long, 4> {
        const Region& R = regions[S.region];
        Op4 o = row_op(R, S.col, i, 0, false);
        if (S.ncols == 2) {
            const Op4 o2 = row_op(R, S.col + 1, i, 0, false);
            o.u *= o2.u; o.d *= o2.d; o.r = o2.r;
        }
        return {o.u, o.l, o.d, o.r};
    };
    // scratch maxima over every strip row (the chains and the closings use the same rows)
    // Layered rows (real double-layer lattices): a site row contracts the ket tensor T (or O T at
    // an operator site) and the bra tensor T one after the other instead of the double-layer
    // E = sum_p (O T)_p T_p; the same sums in another order, with about a fifth of the flops of
    // the E contraction at D = 5.
    const bool layered = !L->cplx && !L->single && !L->hb;
    // a site row of a one-column strip takes the layered route when both of its pair
    // contractions (down: legs u, l against d, r; up: d, l against u, r) fit the kernel
    auto layered_site = [&](const Strip& S, int i) {
        if (!layered || S.ncols != 1 || i < 1 || i > regions[S.region].h) return false;
        const Region& R = regions[S.region];
        const auto dd = L->site_dims(R.r0 + i - 1, R.c0 + S.col);
        const int ULd = dd[0] * dd[1], DRd = dd[2] * dd[3], ULu = dd[2] * dd[1], DRu = dd[0] * dd[3];
        if (ULd > 32 || DRd > 32 || ULu > 32 || DRu > 32) return false;
        for (bool f : {false, true})
            if (layer_smem_bytes(d, ULd, DRd, f) > LAYER_SMEM_MAX || layer_smem_bytes(d, ULu, DRu, f) > LAYER_SMEM_MAX)
                return false;
        return true;
    };
    bool any_layered = false;
    size_t fmax = 1, s1max = 1, s2max = 1, o12max = 1, tomax = 1;
    for (auto& S : strips) {
        const Region& R = regions[S.region];
        for (int i = 0; i < R.h + 2; ++i) {
            const View3 Lv = env_site(R, true, S.col, i), Rv = env_site(R, false, S.col + S.ncols - 1, i);
            const auto od = row_dims(S, i);
            const size_t u = od[0], s = Lv.k, v = od[2], t2 = od[3], A = Lv.a, Ap = Lv.b, B = Rv.a, Bp = Rv.b;
            if (od[1] != Lv.k || t2 != (size_t)Rv.k) return fail(BBP_ERR_INVALID, "internal: closing leg mismatch");
            if (i + 1 < R.h + 2) {
                const View3 Ln = env_site(R, true, S.col, i + 1), Rn = env_site(R, false, S.col + S.ncols - 1, i + 1);
                if (Ln.a != Lv.b || Rn.a != Rv.b || row_dims(S, i + 1)[0] != od[2])
                    return fail(BBP_ERR_INVALID, "internal: closing rows do not chain");
            }
            if (S.ncols == 2) {
                const Op4 o = row_op(R, S.col, i, 0, false), o2 = row_op(R, S.col + 1, i, 0, false);
                o12max = std::max(o12max, (size_t)o.u * o2.u * o.l * o.d * o2.d * o2.r);
            }
            fmax = std::max({fmax, A * u * B, Ap * v * Bp});
            if (layered_site(S, i)) {  // O T and T of an operator site in this row
                const auto dd = L->site_dims(R.r0 + i - 1, R.c0 + S.col);
                tomax = std::max(tomax, 2 * (size_t)d * dd[0] * dd[1] * dd[2] * dd[3]);
                any_layered = true;
            }
            s1max = std::max({s1max, u * B * s * Ap, v * Bp * s * A});     // G1 (down), X1 (up)
            s2max = std::max({s2max, B * Ap * v * t2, Bp * A * u * t2});   // G2 (down), X2 (up)
            if (i >= 1) S.chain += A * u * B;                              // T_i, i = 1..h+1
            if (i >= 2) S.chain += A * u * B;                              // G_i, i = 2..h+1
        }
    }
    struct Lane {
        size_t F[2], S1, S2, EO[2], O12, TO[2];
    };
    const size_t lane_elems = 2 * fmax + s1max + s2max + (L->single ? 0 : 2 * (size_t)K4max) + o12max +
                              (any_layered ? 2 * tomax : 0);
    // device memory for the read-out's scratch: up to a quarter of what is free (at least 1 GB,
    // at most 16 GB), half of it for lanes, half for the strips' environments
    size_t mem_free = 0, mem_total = 0;
    CKR(cudaMemGetInfo(&mem_free, &mem_total));
    const size_t budget = std::max<size_t>((size_t)1 << 30, std::min<size_t>((size_t)16 << 30, mem_free / 4));
    const size_t nlanes =
        std::max<size_t>(2, std::min<size_t>(std::max<size_t>(2, nclos), budget / 2 / std::max<size_t>(1, lane_elems * ss)));
    const size_t chain_budget = budget / 2 / (size_t)ss;
    // waves of strips: two lanes per strip for its chains, environments within the budget
    std::vector<std::vector<int>> waves;
    size_t chain_cap = 1;
    {
        std::vector<int> cur;
        size_t tot = 0;
        for (int k = 0; k < (int)strips.size(); ++k) {
            if (!cur.empty() && (2 * (cur.size() + 1) > nlanes || tot + strips[k].chain > chain_budget)) {
                waves.push_back(cur);
                cur.clear();
                tot = 0;
            }
            cur.push_back(k);
            tot += strips[k].chain;
            chain_cap = std::max(chain_cap, tot);
        }
        if (!cur.empty()) waves.push_back(cur);
    }
    const size_t chain_base = elem_alloc(chain_cap);
    // Closings in FP32 arithmetic (tensor-core lattices unless keep_fp64): every environment is
    // rescaled by a power of two after it is formed (exact), its exponent kept on the device
    // and restored in the FP64 inner products, so that no FP32 intermediate overflows however
    // many rows a strip has.
    const bool f32c = L->mixed && !ds.keep_fp64;
    size_t exp_cap = 1;
    for (const auto& wave : waves) {
        size_t e = 0;
        for (int k : wave) e += 2 * (size_t)(regions[strips[k].region].h + 2);
        exp_cap = std::max(exp_cap, e);
    }
    const size_t exp_base = pr.arena_alloc(exp_cap * sizeof(int));
    auto eptr = [&](size_t byte_off) { return (const int*)P(byte_off); };
    std::vector<Lane> lanes(nlanes);
    for (auto& ln : lanes) {
        ln.F[0] = elem_alloc(fmax); ln.F[1] = elem_alloc(fmax);
        ln.S1 = elem_alloc(s1max); ln.S2 = elem_alloc(s2max);
        if (!L->single) {
            ln.EO[0] = elem_alloc(K4max);
            ln.EO[1] = elem_alloc(K4max);
        }
        ln.O12 = elem_alloc(o12max);
        if (any_layered) {
            ln.TO[0] = elem_alloc(tomax);
            ln.TO[1] = elem_alloc(tomax);
        }
    }
    // operators (impurity tensors) of every closing, each in its own slab: uploaded once
    // before the read-out runs, whichever wave of lanes uses them
    std::vector<std::pair<size_t, std::vector<double>>> uploads;
    {
        std::vector<RatioTask> rt(n_terms);
        for (int t = 0; t < n_terms; ++t) {
            RatioTask& r = rt[t];
            r = RatioTask{};
            if (tplan[t].parts.size() > 4) return fail(BBP_ERR_INVALID, "internal: more than four operator parts");
            r.nparts = (int)tplan[t].parts.size();
            for (int k = 0; k < r.nparts; ++k) {
                r.part[k] = tplan[t].parts[k].first;
                r.c_re[k] = tplan[t].parts[k].second.real();
                r.c_im[k] = tplan[t].parts[k].second.imag();
            }
            r.denom = tplan[t].denom;
        }
        std::vector<double> words(rt.size() * sizeof(RatioTask) / sizeof(double));
        if (!rt.empty()) std::memcpy(words.data(), rt.data(), rt.size() * sizeof(RatioTask));
        uploads.push_back({ratio_tasks / (size_t)ss, words});  // byte offsets are 256-aligned
    }
    std::vector<std::array<size_t, 2>> opoff(nclos, std::array<size_t, 2>{0, 0});
    for (size_t ci = 0; ci < nclos; ++ci)
        for (size_t k = 0; k < closings[ci].pos.size(); ++k) {
            const std::vector<double>& v = closings[ci].ops[k];
            // complex operators take two doubles per element in the Hermitian basis
            opoff[ci][k] = elem_alloc(L->cplx ? v.size() / 2 : v.size());
            uploads.push_back({opoff[ci][k], v});
        }
    // layered operator rows: [O; 1], so that one contraction writes O T and a copy of T side by
    // side in the lane (the layered kernel finds the bra tensor at a fixed offset from the ket,
    // and the read-out's buffers and the lattice's are placed independently)
    std::vector<std::array<size_t, 2>> opaug(nclos, std::array<size_t, 2>{0, 0});
    if (any_layered)
        for (size_t ci = 0; ci < nclos; ++ci)
            for (size_t k = 0; k < closings[ci].pos.size(); ++k) {
                std::vector<double> v = closings[ci].ops[k];
                if (v.size() != (size_t)d * d) continue;  // real d x d operators only
                v.resize(2 * (size_t)d * d, 0.0);
                for (int p = 0; p < d; ++p) v[(size_t)(d + p) * d + p] = 1.0;
                opaug[ci][k] = elem_alloc(v.size());
                uploads.push_back({opaug[ci][k], v});
            }

    // strip row i's operator, E^O at the sites listed in subs (local (row, col), offset); a
    // column pair is fused into o12 first
    bool leg_error = false;
    auto strip_op = [&](const Strip& S, int i, const std::vector<std::pair<std::pair<int, int>, size_t>>& subs,
                        size_t o12, std::vector<FuseTask>& ft, long long& fmx) -> Op4 {
        const Region& R = regions[S.region];
        auto op_at = [&](int c) {
            for (auto& sb : subs)
                if (sb.first.first == i - 1 && sb.first.second == c) return row_op(R, c, i, sb.second, true);
            return row_op(R, c, i, 0, false);
        };
        Op4 o = op_at(S.col);
        if (S.ncols == 2) {
            const Op4 o2 = op_at(S.col + 1);
            FuseTask f{};
            f.A = P(o.off * ss); f.B = P(o2.off * ss); f.out = P(o12 * ss);
            f.u1 = o.u; f.l1 = o.l; f.d1 = o.d; f.m = o.r; f.u2 = o2.u; f.d2 = o2.d; f.r2 = o2.r;
            f.a_u = o.su; f.a_l = o.sl; f.a_d = o.sd; f.a_r = o.sr;
            f.b_u = o2.su; f.b_l = o2.sl; f.b_d = o2.sd; f.b_r = o2.sr;
            if (o.r != o2.l) leg_error = true;
            ft.push_back(f);
            fmx = std::max(fmx, (long long)o.u * o2.u * o.l * o.d * o2.d * o2.r);
            o = op_contig(o12, o.u * o2.u, o.l, o.d * o2.d, o2.r);
        }
        return o;
    };
    // one row downwards: Fout[Ap][v][Bp] = sum Fin[A][W][B] L[A][s][Ap] O[W][s][v][t2] R[B][t2][Bp]
    // through G1[W][B][s][Ap] and G2[B][Ap][v][t2]
    auto row_down = [&](size_t Fin, size_t Fout, const View3& Lv, const Op4& o, const View3& Rv, const Lane& ln,
                        std::vector<GTask>& g1, std::vector<GTask>& g2, std::vector<GTask>& g3) {
        const long long A_ = Lv.a, Wd = o.u, B_ = Rv.a, s = Lv.k, Ap = Lv.b, v = o.d, t2 = o.r, Bp = Rv.b;
        GTask a{};
        a.A = P(Fin * ss); a.B = P(Lv.off * ss); a.C = P(ln.S1 * ss);
        a.M1 = (int)Wd; a.M2 = (int)B_; a.K1 = 1; a.K2 = (int)A_; a.N1 = (int)s; a.N2 = (int)Ap;
        a.a_m1 = B_; a.a_m2 = 1; a.a_k2 = Wd * B_;
        a.b_k2 = Lv.sa; a.b_n1 = Lv.sk; a.b_n2 = Lv.sb;
        a.c_m1 = B_ * s * Ap; a.c_m2 = s * Ap; a.c_n1 = Ap; a.c_n2 = 1;
        g1.push_back(a);
        GTask b{};
        b.A = P(ln.S1 * ss); b.B = P(o.off * ss); b.C = P(ln.S2 * ss);
        b.M1 = (int)B_; b.M2 = (int)Ap; b.K1 = (int)Wd; b.K2 = (int)s; b.N1 = (int)v; b.N2 = (int)t2;
        b.a_m1 = s * Ap; b.a_m2 = 1; b.a_k1 = B_ * s * Ap; b.a_k2 = Ap;
        b.b_k1 = o.su; b.b_k2 = o.sl; b.b_n1 = o.sd; b.b_n2 = o.sr;
        b.c_m1 = Ap * v * t2; b.c_m2 = v * t2; b.c_n1 = t2; b.c_n2 = 1;
        g2.push_back(b);
        GTask c{};
        c.A = P(ln.S2 * ss); c.B = P(Rv.off * ss); c.C = P(Fout * ss);
        c.M1 = (int)Ap; c.M2 = (int)v; c.K1 = (int)B_; c.K2 = (int)t2; c.N1 = 1; c.N2 = (int)Bp;
        c.a_m1 = v * t2; c.a_m2 = t2; c.a_k1 = Ap * v * t2; c.a_k2 = 1;
        c.b_k1 = Rv.sa; c.b_k2 = Rv.sk; c.b_n2 = Rv.sb;
        c.c_m1 = v * Bp; c.c_m2 = Bp; c.c_n2 = 1;
        g3.push_back(c);
    };
    // one row upwards: Gout[A][W][B] = sum L[A][s][Ap] O[W][s][v][t2] R[B][t2][Bp] Gin[Ap][v][Bp]
    // through X1[v][Bp][s][A] and X2[Bp][A][W][t2] (row_down with the roles of the legs swapped)
    auto row_up = [&](size_t Gin, size_t Gout, const View3& Lv, const Op4& o, const View3& Rv, const Lane& ln,
                      std::vector<GTask>& g1, std::vector<GTask>& g2, std::vector<GTask>& g3) {
        const long long A_ = Lv.a, Wd = o.u, B_ = Rv.a, s = Lv.k, Ap = Lv.b, v = o.d, t2 = o.r, Bp = Rv.b;
        GTask a{};
        a.A = P(Gin * ss); a.B = P(Lv.off * ss); a.C = P(ln.S1 * ss);
        a.M1 = (int)v; a.M2 = (int)Bp; a.K1 = 1; a.K2 = (int)Ap; a.N1 = (int)s; a.N2 = (int)A_;
        a.a_m1 = Bp; a.a_m2 = 1; a.a_k2 = v * Bp;
        a.b_k2 = Lv.sb; a.b_n1 = Lv.sk; a.b_n2 = Lv.sa;
        a.c_m1 = Bp * s * A_; a.c_m2 = s * A_; a.c_n1 = A_; a.c_n2 = 1;
        g1.push_back(a);
        GTask b{};
        b.A = P(ln.S1 * ss); b.B = P(o.off * ss); b.C = P(ln.S2 * ss);
        b.M1 = (int)Bp; b.M2 = (int)A_; b.K1 = (int)v; b.K2 = (int)s; b.N1 = (int)Wd; b.N2 = (int)t2;
        b.a_m1 = s * A_; b.a_m2 = 1; b.a_k1 = Bp * s * A_; b.a_k2 = A_;
        b.b_k1 = o.sd; b.b_k2 = o.sl; b.b_n1 = o.su; b.b_n2 = o.sr;
        b.c_m1 = A_ * Wd * t2; b.c_m2 = Wd * t2; b.c_n1 = t2; b.c_n2 = 1;
        g2.push_back(b);
        GTask c{};
        c.A = P(ln.S2 * ss); c.B = P(Rv.off * ss); c.C = P(Gout * ss);
        c.M1 = (int)A_; c.M2 = (int)Wd; c.K1 = (int)Bp; c.K2 = (int)t2; c.N1 = 1; c.N2 = (int)B_;
        c.a_m1 = Wd * t2; c.a_m2 = t2; c.a_k1 = A_ * Wd * t2; c.a_k2 = 1;
        c.b_k1 = Rv.sb; c.b_k2 = Rv.sk; c.b_n2 = Rv.sa;
        c.c_m1 = Wd * B_; c.c_m2 = B_; c.c_n2 = 1;
        g3.push_back(c);
    };
    // Layered rows: g1 and g3 as in row_down / row_up, and between them one layered pair
    // contraction (GTask::layer_d) with the ket tensor tk (T, or O T at an operator site) and
    // the bra tensor T in place of the contraction with E.  Downwards the pairs are (B, Ap),
    // the contracted double legs (u u'), (l l') of G1 and the free ones (d d'), (r r') of G2;
    // upwards the pairs are (Bp, A), contracted (d d'), (l l') of X1, free (u u'), (r r') of X2.
    auto row_down_layered = [&](size_t Fin, size_t Fout, const View3& Lv, const View3& Rv, size_t tk, size_t tb,
                                const std::array<int, 4>& dd, const Lane& ln, std::vector<GTask>& g1,
                                std::vector<GTask>& g2, std::vector<GTask>& g3) {
        const long long Du = dd[0], Dl = dd[1], Dd = dd[2], Dr = dd[3], DdDr = Dd * Dr;
        const long long A_ = Lv.a, Wd = Du * Du, B_ = Rv.a, sK = Lv.k, Ap = Lv.b, v = Dd * Dd, t2 = Rv.k, Bp = Rv.b;
        GTask a{};
        a.A = P(Fin * ss); a.B = P(Lv.off * ss); a.C = P(ln.S1 * ss);
        a.M1 = (int)Wd; a.M2 = (int)B_; a.K1 = 1; a.K2 = (int)A_; a.N1 = (int)sK; a.N2 = (int)Ap;
        a.a_m1 = B_; a.a_m2 = 1; a.a_k2 = Wd * B_;
        a.b_k2 = Lv.sa; a.b_n1 = Lv.sk; a.b_n2 = Lv.sb;
        a.c_m1 = B_ * sK * Ap; a.c_m2 = sK * Ap; a.c_n1 = Ap; a.c_n2 = 1;
        g1.push_back(a);
        GTask t{};
        t.A = P(ln.S1 * ss); t.B = P(tk * ss); t.C = P(ln.S2 * ss);
        t.layer_d = d;
        t.tb_off = (long long)tb - (long long)tk;
        t.M1 = (int)B_; t.M2 = (int)Ap; t.K1 = (int)Du; t.K2 = (int)Dl; t.N1 = (int)Dd; t.N2 = (int)Dr;
        t.a_m1 = sK * Ap; t.a_m2 = 1; t.a_k1 = B_ * sK * Ap; t.a_k2 = Ap;       // G1[W][B][s][Ap]
        t.b_k1 = Dl * DdDr; t.b_k2 = DdDr; t.b_n1 = Dr; t.b_n2 = 1;              // T[p][u][l][d][r]
        t.c_m1 = Ap * v * t2; t.c_m2 = v * t2; t.c_n1 = t2; t.c_n2 = 1;          // G2[B][Ap][v][t2]
        g2.push_back(t);
        GTask c{};
        c.A = P(ln.S2 * ss); c.B = P(Rv.off * ss); c.C = P(Fout * ss);
        c.M1 = (int)Ap; c.M2 = (int)v; c.K1 = (int)B_; c.K2 = (int)t2; c.N1 = 1; c.N2 = (int)Bp;
        c.a_m1 = v * t2; c.a_m2 = t2; c.a_k1 = Ap * v * t2; c.a_k2 = 1;
        c.b_k1 = Rv.sa; c.b_k2 = Rv.sk; c.b_n2 = Rv.sb;
        c.c_m1 = v * Bp; c.c_m2 = Bp; c.c_n2 = 1;
        g3.push_back(c);
    };
    auto row_up_layered = [&](size_t Gin, size_t Gout, const View3& Lv, const View3& Rv, size_t tk, size_t tb,
                              const std::array<int, 4>& dd, const Lane& ln, std::vector<GTask>& g1,
                              std::vector<GTask>& g2, std::vector<GTask>& g3) {
        const long long Du = dd[0], Dl = dd[1], Dd = dd[2], Dr = dd[3], DdDr = Dd * Dr;
        const long long A_ = Lv.a, Wd = Du * Du, B_ = Rv.a, sK = Lv.k, Ap = Lv.b, v = Dd * Dd, t2 = Rv.k, Bp = Rv.b;
        GTask a{};
        a.A = P(Gin * ss); a.B = P(Lv.off * ss); a.C = P(ln.S1 * ss);
        a.M1 = (int)v; a.M2 = (int)Bp; a.K1 = 1; a.K2 = (int)Ap; a.N1 = (int)sK; a.N2 = (int)A_;
        a.a_m1 = Bp; a.a_m2 = 1; a.a_k2 = v * Bp;
        a.b_k2 = Lv.sb; a.b_n1 = Lv.sk; a.b_n2 = Lv.sa;
        a.c_m1 = Bp * sK * A_; a.c_m2 = sK * A_; a.c_n1 = A_; a.c_n2 = 1;
        g1.push_back(a);
        GTask t{};
        t.A = P(ln.S1 * ss); t.B = P(tk * ss); t.C = P(ln.S2 * ss);
        t.layer_d = d;
        t.tb_off = (long long)tb - (long long)tk;
        t.M1 = (int)Bp; t.M2 = (int)A_; t.K1 = (int)Dd; t.K2 = (int)Dl; t.N1 = (int)Du; t.N2 = (int)Dr;
        t.a_m1 = sK * A_; t.a_m2 = 1; t.a_k1 = Bp * sK * A_; t.a_k2 = A_;       // X1[v][Bp][s][A]
        t.b_k1 = Dr; t.b_k2 = DdDr; t.b_n1 = Dl * DdDr; t.b_n2 = 1;            // T[p][u][l][d][r]
        t.c_m1 = A_ * Wd * t2; t.c_m2 = Wd * t2; t.c_n1 = t2; t.c_n2 = 1;        // X2[Bp][A][W][t2]
        g2.push_back(t);
        GTask c{};
        c.A = P(ln.S2 * ss); c.B = P(Rv.off * ss); c.C = P(Gout * ss);
        c.M1 = (int)A_; c.M2 = (int)Wd; c.K1 = (int)Bp; c.K2 = (int)t2; c.N1 = 1; c.N2 = (int)B_;
        c.a_m1 = Wd * t2; c.a_m2 = t2; c.a_k1 = A_ * Wd * t2; c.a_k2 = 1;
        c.b_k1 = Rv.sb; c.b_k2 = Rv.sk; c.b_n2 = Rv.sa;
        c.c_m1 = Wd * B_; c.c_m2 = B_; c.c_n2 = 1;
        g3.push_back(c);
    };
    auto is_layered = [&](const Strip& S, int i) { return layered_site(S, i); };
    auto site_T = [&](const Strip& S, int i) {
        const Region& R = regions[S.region];
        return L->T_off[L->tensor_index(R.r0 + i - 1, R.c0 + S.col)];
    };
    auto site_dd = [&](const Strip& S, int i) {
        const Region& R = regions[S.region];
        return L->site_dims(R.r0 + i - 1, R.c0 + S.col);
    };
    auto fuse_step = [&](std::vector<FuseTask>& ft, long long fmx) {
        if (ft.empty()) return;
        Step s;
        s.kind = ST_FUSE;
        s.first = pr.fus.size();
        s.count = (int)ft.size();
        s.n = fmx;
        pr.fus.insert(pr.fus.end(), ft.begin(), ft.end());
        pr.steps.push_back(s);
        ft.clear();
    };
    auto env_scalars = [&](const Strip& S, int i) {  // scalars of T_i / G_i
        const Region& R = regions[S.region];
        const View3 Lv = env_site(R, true, S.col, i), Rv = env_site(R, false, S.col + S.ncols - 1, i);
        return (size_t)Lv.a * (size_t)row_dims(S, i)[0] * (size_t)Rv.a;
    };

    pr.gc_f32 = f32c;
    for (const auto& wave : waves) {
        // environments of this wave's strips, in the shared chain slab
        size_t at = chain_base, eat = exp_base;
        int hmax = 0;
        for (int k : wave) {
            Strip& S = strips[k];
            const int h = regions[S.region].h;
            hmax = std::max(hmax, h);
            S.T.assign(h + 2, 0);
            S.G.assign(h + 2, 0);
            S.eT.assign(h + 2, 0);
            S.eG.assign(h + 2, 0);
            for (int i = 0; i < h + 2; ++i) {
                S.eT[i] = eat + (size_t)i * sizeof(int);
                S.eG[i] = eat + (size_t)(h + 2 + i) * sizeof(int);
            }
            eat += 2 * (size_t)(h + 2) * sizeof(int);
            for (int i = 1; i <= h + 1; ++i) {
                S.T[i] = at;
                at += env_scalars(S, i);
            }
            for (int i = 2; i <= h + 1; ++i) {
                S.G[i] = at;
                at += env_scalars(S, i);
            }
        }
        // the chains: step j takes top row j and bottom row h+1-j of every strip
        for (int j = 0; j <= hmax + 1; ++j) {
            std::vector<FuseTask> ft;
            long long fmx = 1;
            std::vector<GTask> g1, g2, g2l, g3;
            std::vector<DotTask> p2;
            for (size_t q = 0; q < wave.size(); ++q) {
                const Strip& S = strips[wave[q]];
                const Region& R = regions[S.region];
                const int h = R.h;
                const Lane& top = lanes[2 * q];
                const Lane& bot = lanes[2 * q + 1];
                if (j <= h) {
                    if (is_layered(S, j)) {
                        row_down_layered(S.T[j], S.T[j + 1], env_site(R, true, S.col, j),
                                         env_site(R, false, S.col, j), site_T(S, j), site_T(S, j), site_dd(S, j),
                                         top, g1, g2l, g3);
                    } else {
                        const Op4 o = strip_op(S, j, {}, top.O12, ft, fmx);
                        row_down(j == 0 ? L->one_off : S.T[j], S.T[j + 1], env_site(R, true, S.col, j),
                                 o, env_site(R, false, S.col + S.ncols - 1, j), top, g1, g2, g3);
                    }
                    DotTask t{};
                    t.A = P(S.T[j + 1] * ss); t.out = P(S.eT[j + 1]); t.n = (long long)env_scalars(S, j + 1);
                    t.ea = j == 0 ? nullptr : eptr(S.eT[j]);
                    p2.push_back(t);
                }
                const int ib = h + 1 - j;
                if (ib >= 2) {
                    if (is_layered(S, ib)) {
                        row_up_layered(S.G[ib + 1], S.G[ib], env_site(R, true, S.col, ib),
                                       env_site(R, false, S.col, ib), site_T(S, ib), site_T(S, ib), site_dd(S, ib),
                                       bot, g1, g2l, g3);
                    } else {
                        const Op4 o = strip_op(S, ib, {}, bot.O12, ft, fmx);
                        row_up(ib == h + 1 ? L->one_off : S.G[ib + 1], S.G[ib], env_site(R, true, S.col, ib), o,
                               env_site(R, false, S.col + S.ncols - 1, ib), bot, g1, g2, g3);
                    }
                    DotTask t{};
                    t.A = P(S.G[ib] * ss); t.out = P(S.eG[ib]); t.n = (long long)env_scalars(S, ib);
                    t.ea = ib == h + 1 ? nullptr : eptr(S.eG[ib + 1]);
                    p2.push_back(t);
                }
            }
            fuse_step(ft, fmx);
            pr.gc_step(g1);
            pr.gc_step(g2);
            pr.layer_step(g2l);
            pr.gc_step(g3);
            if (f32c) pr.dot_step(p2, true);
        }
        // the strips' norms, then their closings, nlanes at a time
        std::vector<DotTask> dts;
        std::vector<int> cl;
        for (int k : wave) {
            const Strip& S = strips[k];
            const int h = regions[S.region].h;
            DotTask t{};
            t.A = P(S.T[h + 1] * ss); t.B = P(S.G[h + 1] * ss); t.out = P((results + S.norm) * ss);
            t.n = (long long)env_scalars(S, h + 1);
            if (f32c) {
                t.ea = eptr(S.eT[h + 1]);
                t.eb = eptr(S.eG[h + 1]);
            }
            dts.push_back(t);
            cl.insert(cl.end(), S.clos.begin(), S.clos.end());
        }
        pr.dot_step(dts);
        std::vector<int> strip_of(nclos, -1);
        for (int k : wave)
            for (int ci : strips[k].clos) strip_of[ci] = k;
        for (size_t w0 = 0; w0 < cl.size(); w0 += nlanes) {
            const size_t w1 = std::min(cl.size(), w0 + nlanes);
            // E^O for the operator sites of these closings
            std::vector<DLTask> dlt;
            std::vector<GTask> otk;
            long long dlmax = 1;
            std::vector<int> i0(w1 - w0), i1(w1 - w0);
            int nrows = 0;
            for (size_t q = w0; q < w1; ++q) {
                const int ci = cl[q];
                const Closing& C = closings[ci];
                const Region& R = regions[C.region];
                const Lane& ln = lanes[q - w0];
                i0[q - w0] = 1 << 30;
                i1[q - w0] = -1;
                for (size_t k = 0; k < C.pos.size(); ++k) {
                    i0[q - w0] = std::min(i0[q - w0], C.pos[k].first + 1);
                    i1[q - w0] = std::max(i1[q - w0], C.pos[k].first + 1);
                    if (L->single) continue;  // the impurity tensor is E^O itself
                    const int r = R.r0 + C.pos[k].first, c = R.c0 + C.pos[k].second;
                    const auto dd = L->site_dims(r, c);
                    if (is_layered(strips[strip_of[ci]], C.pos[k].first + 1)) {
                        // layered row: the ket tensor O T and the bra tensor T,
                        //   TO[p'][x] = sum_p [O; 1][p'][p] T[p][x], p' < 2d
                        const long long vol = (long long)dd[0] * dd[1] * dd[2] * dd[3];
                        if (!opaug[ci][k]) return fail(BBP_ERR_INVALID, "internal: layered operator missing");
                        GTask t{};
                        t.A = P(opaug[ci][k] * ss); t.B = P(L->T_off[L->tensor_index(r, c)] * ss);
                        t.C = P(ln.TO[k] * ss);
                        t.M1 = 1; t.M2 = 2 * d; t.K1 = 1; t.K2 = d; t.N1 = 1; t.N2 = (int)vol;
                        t.a_m2 = d; t.a_k2 = 1; t.b_k2 = vol; t.b_n2 = 1; t.c_m2 = vol; t.c_n2 = 1;
                        otk.push_back(t);
                        continue;
                    }
                    DLTask t{};
                    t.T = P(L->T_off[L->tensor_index(r, c)] * ss);
                    t.E = P(ln.EO[k] * ss);
                    t.O = P(opoff[ci][k] * ss);
                    t.d = d; t.Du = dd[0]; t.Dl = dd[1]; t.Dd = dd[2]; t.Dr = dd[3];
                    t.hb = L->hb ? 1 : 0;
                    dlt.push_back(t);
                    dlmax = std::max(dlmax, (long long)dd[0] * dd[0] * dd[1] * dd[1] * dd[2] * dd[2] * dd[3] * dd[3]);
                }
                nrows = std::max(nrows, i1[q - w0] - i0[q - w0] + 1);
            }
            if (!dlt.empty()) {
                Step s;
                s.kind = ST_DL;
                s.first = pr.dl.size();
                s.count = (int)dlt.size();
                s.n = dlmax;
                s.aux2 = L->hb ? 1 : 0;
                pr.dl.insert(pr.dl.end(), dlt.begin(), dlt.end());
                pr.steps.push_back(s);
            }
            pr.gc_step(otk);
            for (int rr = 0; rr < nrows; ++rr) {
                std::vector<FuseTask> ft;
                long long fmx = 1;
                std::vector<GTask> g1, g2, g2l, g3;
                for (size_t q = w0; q < w1; ++q) {
                    const int i = i0[q - w0] + rr;
                    if (i > i1[q - w0]) continue;
                    const int ci = cl[q];
                    const Closing& C = closings[ci];
                    const Strip& S = strips[strip_of[ci]];
                    const Region& R = regions[S.region];
                    const Lane& ln = lanes[q - w0];
                    const size_t Fin = rr == 0 ? S.T[i] : ln.F[(rr - 1) % 2];
                    if (is_layered(S, i)) {
                        size_t tk = site_T(S, i), tb = tk;
                        for (size_t k = 0; k < C.pos.size(); ++k)
                            if (C.pos[k].first == i - 1 && C.pos[k].second == S.col) {
                                const auto dd = site_dd(S, i);
                                tk = ln.TO[k];
                                tb = tk + (size_t)d * dd[0] * dd[1] * dd[2] * dd[3];
                                break;
                            }
                        row_down_layered(Fin, ln.F[rr % 2], env_site(R, true, S.col, i), env_site(R, false, S.col, i),
                                         tk, tb, site_dd(S, i), ln, g1, g2l, g3);
                        continue;
                    }
                    std::vector<std::pair<std::pair<int, int>, size_t>> subs;
                    for (size_t k = 0; k < C.pos.size(); ++k)
                        subs.push_back({C.pos[k], L->single ? opoff[ci][k] : ln.EO[k]});
                    const Op4 o = strip_op(S, i, subs, ln.O12, ft, fmx);
                    row_down(Fin, ln.F[rr % 2], env_site(R, true, S.col, i), o,
                             env_site(R, false, S.col + S.ncols - 1, i), ln, g1, g2, g3);
                }
                fuse_step(ft, fmx);
                pr.gc_step(g1);
                pr.gc_step(g2);
                pr.layer_step(g2l);
                pr.gc_step(g3);
            }
            // N_O = <F after the closing's last row, G below it>
            for (size_t q = w0; q < w1; ++q) {
                const int ci = cl[q];
                const Strip& S = strips[strip_of[ci]];
                const int last = i1[q - w0], nr = last - i0[q - w0] + 1;
                DotTask t{};
                t.A = P(lanes[q - w0].F[(nr - 1) % 2] * ss);
                t.B = P(S.G[last + 1] * ss);
                t.out = P((results + ci) * ss);
                t.n = (long long)env_scalars(S, last + 1);
                if (f32c) {
                    t.ea = eptr(S.eT[i0[q - w0]]);
                    t.eb = eptr(S.eG[last + 1]);
                }
                dts.push_back(t);
            }
            pr.dot_step(dts);
        }
    }
    if (leg_error) return fail(BBP_ERR_INVALID, "internal: column pair leg mismatch");

    // ---- check, allocate, relocate, upload, run
    pr.parent = &L->sweep;
    pr.split = split;
    {
        const std::string v = pr.validate();
        if (!v.empty()) return fail(BBP_ERR_INVALID, "internal read-out plan check: " + v);
    }
    const size_t ro_bytes = pr.arena_used - split;
    char* ro = nullptr;
    cudaStream_t st = L->stream;
    CKR(cudaMallocAsync((void**)&ro, ro_bytes, st));
    struct Guard {  // stream-ordered release after the read-out's last kernel
        char* p;
        Program* pr;
        cudaStream_t st;
        ~Guard() {
            pr->free_all(st);
            cudaFreeAsync(p, st);
        }
    } guard{ro, &pr, st};
    pr.relocate(L->arena, split, ro);
    pr.status = L->d_status;
    if (tc_env) CKR(pr.encode_maps(L->arena, split, ro));
    CKR(pr.upload_tasks(st));
    CKR(cudaMemsetAsync(ro, 0, ro_bytes, st));
    for (auto& u : uploads) {
        const size_t bytes = u.second.size() * sizeof(double);
        CKR(cudaMemcpyAsync(ro + (u.first * ss - split), u.second.data(), bytes, cudaMemcpyHostToDevice, st));
    }
    if (!pr.loop_descs.empty() && ds.launch_mode == 0) {
        // one graph: each fit loop is a conditional WHILE node that stops when its fits
        // have converged, instead of launching every loop body its maximum number of times
        // (launch_mode 1: the kernels one by one, as for the sweep)
        CKR(pr.build_graph(st, nullptr, ds.seed));
        CKR(cudaGraphLaunch(pr.exec, st));
    } else {
        CKR(pr.init_loops(st, false, nullptr));
        CKR(pr.launch_all(st, nullptr, ds.seed));
    }
    // <O> = N_O / N_I for every term on the device (FP64), then one copy of the results
    char* rbase = ro - split;  // arena byte offset -> address in the read-out buffer
    CKR(launch_ratio((const RatioTask*)(rbase + ratio_tasks), n_terms, rbase + results * ss, L->cplx,
                     (double*)(rbase + ratio_out), (int*)(rbase + ratio_status), st));
    std::vector<double> res((size_t)n_terms * 2);
    CKR(cudaMemcpyAsync(res.data(), rbase + ratio_out, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    int status = 0, tc_status = 0, ratio_st = 0;
    CKR(cudaMemcpyAsync(&status, L->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaMemcpyAsync(&ratio_st, rbase + ratio_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (tc_env) CKR(cudaMemcpyAsync(&tc_status, L->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (tc_status) return fail(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its bound");
    L->readout_kernels += pr.kernel_count() + 1;
    L->readout_flops += pr.static_flops + pr.gated_flops;
    if (status) return fail(BBP_ERR_NUMERIC, "an environment column has zero or non-finite norm");
    if (ratio_st) return fail(BBP_ERR_NUMERIC, "the closed network vanished");
    for (int t = 0; t < n_terms; ++t) {
        out_re[t] = res[2 * (size_t)t];
        if (out_im) out_im[t] = res[2 * (size_t)t + 1];
    }
    return BBP_OK;
} catch (...) {
    return abi_error();
}

// Read-out over several partitions of one lattice (Sec. "The blockBP algorithm": observables are
// accurate near a block's centre, so every bond is read from a partition whose blocks hold it
// away from their edges).  Each term goes to the lattice in which its sites lie deepest inside
// one block: the smallest distance of any of its sites to that block's edges (a pair split
// between two blocks scores -1), the first lattice on a tie; then one bbp_expect per lattice.
extern "C" int bbp_expect_centred(bbp_lattice* const* lats, int n_lats, const bbp_term* terms, int n_terms,
                                  double* out_re, double* out_im, int* chosen) try {
    if (!lats || n_lats < 1) return fail(BBP_ERR_INVALID, "expect_centred: no lattices");
    if (n_terms < 0 || (n_terms > 0 && (!terms || !out_re))) return fail(BBP_ERR_INVALID, "bad term arguments");
    for (int k = 0; k < n_lats; ++k) {
        if (!lats[k]) return fail(BBP_ERR_INVALID, "expect_centred: a lattice is NULL");
        const bbp_lattice_desc& a = lats[k]->desc;
        const bbp_lattice_desc& b = lats[0]->desc;
        if (a.boundary != BBP_OBC || a.Lx != b.Lx || a.Ly != b.Ly || a.d != b.d)
            return fail(BBP_ERR_INVALID, "expect_centred: OBC partitions of one lattice (same Lx, Ly, d) only");
    }
    const int Lx = lats[0]->desc.Lx, Ly = lats[0]->desc.Ly;
    std::vector<int> pick(n_terms, 0);
    for (int t = 0; t < n_terms; ++t) {
        const bbp_term& T = terms[t];
        if (T.nsite < 1 || T.nsite > 2) return fail(BBP_ERR_INVALID, "term must have 1 or 2 sites");
        int best = -2;
        for (int k = 0; k < n_lats; ++k) {
            const bbp_lattice* L = lats[k];
            int score = 1 << 30, blk0 = -1;
            for (int q = 0; q < T.nsite; ++q) {
                const int s = T.site[q];
                if (s < 0 || s >= Lx * Ly) return fail(BBP_ERR_INVALID, "site out of range");
                const int r = s / Lx, c = s % Lx, blk = L->block_of(r, c);
                int r0, c0, h, w;
                L->block_origin(blk, r0, c0);
                L->block_size(blk, h, w);
                const int dist = std::min(std::min(r - r0, r0 + h - 1 - r), std::min(c - c0, c0 + w - 1 - c));
                if (q == 0) blk0 = blk;
                score = blk != blk0 ? -1 : std::min(score, dist);
            }
            if (score > best) {
                best = score;
                pick[t] = k;
            }
        }
        if (chosen) chosen[t] = pick[t];
    }
    for (int k = 0; k < n_lats; ++k) {
        std::vector<bbp_term> sub;
        std::vector<int> idx;
        for (int t = 0; t < n_terms; ++t)
            if (pick[t] == k) {
                sub.push_back(terms[t]);
                idx.push_back(t);
            }
        if (sub.empty()) continue;
        std::vector<double> re(sub.size()), im(sub.size());
        const int rc = bbp_expect(lats[k], sub.data(), (int)sub.size(), re.data(), im.data());
        if (rc < 0) return rc;
        for (size_t i = 0; i < idx.size(); ++i) {
            out_re[idx[i]] = re[i];
            if (out_im) out_im[idx[i]] = im[i];
        }
    }
    return BBP_OK;
} catch (...) {
    return abi_error();
}

// Reduced density matrix of one or two sites (the 2-local RDMs compared between methods by
// their trace distance, Sec. on the transverse Ising model): entry (a, b) = <a|rho|b> is the
// expectation of the matrix unit |b><a| (a product of single-site units for two sites), read
// out in one bbp_expect call, so that Tr(rho O) = <O> for every operator O on those sites.
extern "C" int bbp_rdm(bbp_lattice* L, int nsite, const int* sites, double* rho_re, double* rho_im) try {
    if (!L) return fail(BBP_ERR_INVALID, "lattice is NULL");
    if (nsite < 1 || nsite > 2 || !sites || !rho_re) return fail(BBP_ERR_INVALID, "rdm: need 1 or 2 sites and rho_re");
    if (L->single) return fail(BBP_ERR_INVALID, "rdm: a single-layer network has no physical leg");
    const int d = L->desc.d, dim = nsite == 1 ? d : d * d;
    // unit[(b * d + a) * d * d ...]: the d x d matrix unit with a 1 at row b, column a
    std::vector<double> units((size_t)d * d * d * d, 0.0);
    for (int b = 0; b < d; ++b)
        for (int a = 0; a < d; ++a) units[((size_t)b * d + a) * d * d + (size_t)b * d + a] = 1.0;
    auto unit = [&](int b, int a) { return units.data() + ((size_t)b * d + a) * d * d; };
    std::vector<bbp_term> terms((size_t)dim * dim);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            bbp_term& t = terms[(size_t)a * dim + b];
            t = bbp_term{};
            t.nsite = nsite;
            for (int k = 0; k < nsite; ++k) {
                // digit k of the row / column index (site 0 is the leading digit)
                const int ak = nsite == 1 ? a : (k == 0 ? a / d : a % d);
                const int bk = nsite == 1 ? b : (k == 0 ? b / d : b % d);
                t.site[k] = sites[k];
                t.op_re[k] = unit(bk, ak);
                t.op_im[k] = nullptr;
            }
        }
    return bbp_expect(L, terms.data(), dim * dim, rho_re, rho_im);
} catch (...) {
    return abi_error();
}
