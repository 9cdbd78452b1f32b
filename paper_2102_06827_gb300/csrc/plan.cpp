// Host planner.  See plan.hpp for the map to the paper.
#include "plan.hpp"

#include <algorithm>
#include <cctype>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <numeric>
#include <set>
#include <sstream>

namespace comet {

// Machine constants of the cost model (GB300): HBM copy bandwidth and dense tensor-core and
// FP64 rates.  Only ratios matter for the choice; they are not reported anywhere.
static const double kHbmBytesPerS = 6.8e12;
static const double kBf16FlopsPerS = 1.67e15;
static const double kF64FlopsPerS = 1.2e12;
static const double kLaunchS = 3e-6;

size_t dtype_size(comet_dtype_t t) { return t == COMET_F32 ? 4 : 8; }

// ------------------------------------------------------------------------------------------
// Parser: lhs (=|+=|-=) [sum_{labels}] factor (* factor)*, factor = number | Name[labels]
// ------------------------------------------------------------------------------------------
namespace {
struct Cursor {
    const char *s;
    size_t i = 0;
    void ws() { while (s[i] && std::isspace((unsigned char)s[i])) ++i; }
    bool eat(char c) { ws(); if (s[i] == c) { ++i; return true; } return false; }
    bool ident(std::string *out) {
        ws();
        size_t j = i;
        if (!(std::isalpha((unsigned char)s[j]) || s[j] == '_')) return false;
        while (std::isalnum((unsigned char)s[j]) || s[j] == '_') ++j;
        out->assign(s + i, j - i);
        i = j;
        return true;
    }
};

bool parse_labels(Cursor &c, std::vector<std::string> *labels, char close) {
    labels->clear();
    if (c.eat(close)) return true;
    for (;;) {
        std::string l;
        if (!c.ident(&l)) return false;
        labels->push_back(l);
        if (c.eat(close)) return true;
        if (!c.eat(',')) return false;
    }
}

bool parse_tensor(Cursor &c, ParsedTensor *t) {
    size_t save = c.i;
    if (!c.ident(&t->name)) { c.i = save; return false; }
    c.ws();
    char open = c.s[c.i];
    if (open != '[' && open != '(') { c.i = save; return false; }
    ++c.i;
    return parse_labels(c, &t->labels, open == '[' ? ']' : ')');
}
}  // namespace

comet_status_t parse_expr(const char *s, ParsedExpr *e, std::string *err) {
    if (!s) return COMET_ERR_NULL;
    Cursor c{s};
    if (!parse_tensor(c, &e->out)) { *err = "left-hand side is not a labelled tensor"; return COMET_ERR_PARSE; }
    c.ws();
    if (c.s[c.i] == '+' && c.s[c.i + 1] == '=') { e->op = 1; c.i += 2; }
    else if (c.s[c.i] == '-' && c.s[c.i + 1] == '=') { e->op = 2; c.i += 2; }
    else if (c.s[c.i] == '=') { e->op = 0; c.i += 1; }
    else { *err = "expected =, += or -="; return COMET_ERR_PARSE; }
    c.ws();
    if (std::strncmp(c.s + c.i, "sum_{", 5) == 0) {
        c.i += 5;
        e->has_sum = true;
        for (;;) {
            c.ws();
            if (c.eat('}')) break;
            std::string l;
            if (!c.ident(&l)) { *err = "bad label in sum_{...}"; return COMET_ERR_PARSE; }
            e->sum_labels.push_back(l);
            c.eat(',');
        }
    }
    e->alpha = 1.0;
    bool any = false;
    for (;;) {
        c.ws();
        ParsedTensor t;
        if (parse_tensor(c, &t)) {
            e->ins.push_back(t);
        } else {
            char *end = nullptr;
            double v = std::strtod(c.s + c.i, &end);
            if (end == c.s + c.i) { *err = "expected a number or a labelled tensor"; return COMET_ERR_PARSE; }
            e->alpha *= v;
            c.i = end - c.s;
        }
        any = true;
        c.ws();
        if (c.s[c.i] == '\0') break;
        if (!c.eat('*')) { *err = "expected *"; return COMET_ERR_PARSE; }
    }
    if (!any || e->ins.empty()) { *err = "no operand on the right-hand side"; return COMET_ERR_PARSE; }
    return COMET_OK;
}

// ------------------------------------------------------------------------------------------
// Transpose engine set-up
// ------------------------------------------------------------------------------------------
namespace {
void fill_radix(Radix *r, const std::vector<int> &dims, const int64_t *ext, const int64_t *s0,
                const int64_t *s1) {
    std::memset(r, 0, sizeof(*r));
    r->n = (int)dims.size();
    uint64_t tot = 1;
    for (int d = 0; d < r->n; ++d) {
        r->ext[d] = (uint32_t)ext[dims[d]];
        r->fd[d] = make_fastdiv(r->ext[d]);
        r->s0[d] = s0[dims[d]];
        r->s1[d] = s1[dims[d]];
        tot *= (uint64_t)ext[dims[d]];
    }
    r->total = (uint32_t)tot;
}

double run_eff(double run_bytes) { return std::min(1.0, run_bytes / 64.0); }
}  // namespace

void setup_xpose(int rank, const int64_t *ext_in, const int64_t *sin_in,
                 const int64_t *sout_in, int elem_bytes, XposeParams *p, int *vec_in,
                 int *vec_out, double *eff, int64_t in_off, int64_t out_off) {
    std::memset(p, 0, sizeof(*p));
    // drop extent-1 dims, then fuse neighbours that are contiguous on both sides
    std::vector<int64_t> ext, si, so;
    for (int d = 0; d < rank; ++d)
        if (ext_in[d] != 1) { ext.push_back(ext_in[d]); si.push_back(sin_in[d]); so.push_back(sout_in[d]); }
    if (ext.empty()) { ext.push_back(1); si.push_back(1); so.push_back(1); }
    // order dims by input stride
    std::vector<int> ord(ext.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return si[a] < si[b]; });
    std::vector<int64_t> e2, i2, o2;
    for (int d : ord) {
        if (!e2.empty() && si[d] == i2.back() * e2.back() && so[d] == o2.back() * e2.back() &&
            (uint64_t)e2.back() * (uint64_t)ext[d] < (1ull << 31)) {
            e2.back() *= ext[d];
        } else {
            e2.push_back(ext[d]); i2.push_back(si[d]); o2.push_back(so[d]);
        }
    }
    int n = (int)e2.size();
    std::vector<int> in_order(n), out_order(n);
    std::iota(in_order.begin(), in_order.end(), 0);
    std::iota(out_order.begin(), out_order.end(), 0);
    std::stable_sort(out_order.begin(), out_order.end(), [&](int a, int b) { return o2[a] < o2[b]; });
    const int64_t target = 64;  // tile edge in elements
    std::vector<int> U, V;
    std::vector<char> used(n, 0);
    int dfi = in_order[0], dfo = out_order[0];
    bool same = (dfi == dfo);
    U.push_back(dfi); used[dfi] = 1;
    int64_t pu = e2[dfi];
    if (!same) { V.push_back(dfo); used[dfo] = 1; }
    int64_t pv = same ? 1 : e2[dfo];
    // extend U along the input order while contiguous in the input
    for (int k = 1; k < n && pu < target; ++k) {
        int d = in_order[k];
        int prev = U.back();
        if (used[d] || i2[d] != i2[prev] * e2[prev] || (uint64_t)pu * e2[d] >= (1ull << 31)) break;
        if (same && o2[d] != o2[prev] * e2[prev]) break;
        U.push_back(d); used[d] = 1; pu *= e2[d];
    }
    if (!same) {
        for (int k = 1; k < n && pv < target; ++k) {
            int d = out_order[k];
            int prev = V.back();
            if (used[d] || o2[d] != o2[prev] * e2[prev] || (uint64_t)pv * e2[d] >= (1ull << 31)) break;
            V.push_back(d); used[d] = 1; pv *= e2[d];
        }
    }
    // copy mode (same stride-1 dim on both sides): V stays empty, R supplies the rows
    std::vector<int> R;
    for (int k = 0; k < n; ++k) if (!used[in_order[k]]) R.push_back(in_order[k]);
    // copy mode with a short shared run (under 128 bytes): a block's rows would otherwise follow
    // the input order only, and each would land as a separate short piece of the output; the
    // row digit nearest to the run in the output comes second, so that a block's rows also
    // form contiguous spans of the output
    if (same && R.size() >= 2 && pu * elem_bytes < 128) {
        size_t best = 1;
        for (size_t k = 2; k < R.size(); ++k) if (o2[R[k]] < o2[R[best]]) best = k;
        if (o2[R[best]] < o2[R[0]]) std::rotate(R.begin() + 1, R.begin() + best, R.begin() + best + 1);
    }
    fill_radix(&p->u, U, e2.data(), i2.data(), o2.data());
    fill_radix(&p->v, V, e2.data(), i2.data(), o2.data());
    fill_radix(&p->r, R, e2.data(), i2.data(), o2.data());
    if (V.empty()) p->v.total = 1;
    if (R.empty()) p->r.total = 1;
    // tile shape: about kXposeTile elements per CTA.  Transposing: 64 along U (reads) and up
    // to 256 along V (writes), the rest from R when both leading runs are short.  Copy mode:
    // up to 256 along U with rows from R; a single fused dim is cut into 4096-element pieces.
    const uint32_t Eu = p->u.total, Ev = p->v.total, Er = p->r.total;
    const uint32_t TAB = 256;
    // 16 KB of elements per tile; COMET_XPOSE_TILE (elements, 1024..16384) overrides it for tuning
    static const uint32_t tile_env = [] {
        const char *s = std::getenv("COMET_XPOSE_TILE");
        const long v = s ? std::strtol(s, nullptr, 10) : 0;
        return (uint32_t)(v >= 1024 && v <= 16384 ? v : 0);
    }();
    const uint32_t TILE = tile_env ? tile_env : elem_bytes == 4 ? (uint32_t)kXposeTile : (uint32_t)kXposeTile / 2;
    const uint32_t W = 16 / elem_bytes;
    // split a run of E into equal pieces of at most maxT, rounded up to a multiple of mult
    auto balanced = [](uint32_t E, uint32_t maxT, uint32_t mult) {
        uint32_t k = (E + maxT - 1) / maxT;
        uint32_t t = (E + k - 1) / k;
        if (mult > 1 && E % mult == 0 && t > mult) {
            const uint32_t up = (t + mult - 1) / mult * mult;
            t = up <= maxT ? up : t / mult * mult;   // never above maxT (the offset tables' size)
        }
        return std::max<uint32_t>(1, std::min(t, E));
    };
    // rounding unit of a tile edge along a leading run (transposing mode): W, or 2 for an FP32
    // run whose first extent is even but not a multiple of 4 (it moves as 8-byte vectors)
    auto edge_mult = [&](const Radix &r) -> uint32_t {
        if (W != 4 || r.n == 0 || r.ext[0] % 2 != 0 || r.ext[0] % 4 == 0 || r.total % 4 == 0) return W;
        return 2;
    };
    const uint32_t mu = edge_mult(p->u), mv = edge_mult(p->v);
    uint32_t tu, tv, tw;
    if (same && R.empty()) {
        tu = Eu > TAB ? std::max<uint32_t>(TAB + 1, std::min<uint32_t>(Eu, TILE)) : Eu;
        tv = 1;
        tw = 1;
    } else if (same) {
        // copy mode keeps no tile in shared memory: rows up to the table size, as long as the
        // grid keeps about 16 blocks per SM
        tu = balanced(Eu, TAB, W);
        tv = 1;
        const uint64_t rows = (uint64_t)Er * ((Eu + tu - 1) / tu);
        const uint64_t want = (rows + 152 * 16 - 1) / (152 * 16);
        tw = (uint32_t)std::min<uint64_t>(Er, std::min<uint64_t>(TAB, std::max<uint64_t>(std::max<uint32_t>(1, TILE / tu), want)));
    } else {
        // both runs at least 64 elements where the extents allow: a leading input run up to 128
        // is kept whole, a longer one is cut into pieces of about 64
        tu = Eu <= 128 ? Eu : balanced(Eu, 64, mu);
        tv = balanced(Ev, std::min<uint32_t>(TAB, std::max<uint32_t>(16, TILE / tu)), mv);
        tw = std::min<uint32_t>(Er, std::min<uint32_t>(TAB, std::max<uint32_t>(1, TILE / (tu * tv))));
    }
    // vector widths: 16-byte accesses when every stride other than the fast digit's is a
    // multiple of the width, the fast digit's extent is too, and the tile edge along the
    // vector direction is a multiple of it; else 8-byte accesses for FP32 on the same terms
    int w = 16 / elem_bytes;
    auto ok_in = [&](int vw) {
        if (in_off % vw || p->u.s0[0] != 1 || p->u.ext[0] % vw || tu % vw) return false;
        for (int d = 1; d < p->u.n; ++d) if (p->u.s0[d] % vw) return false;
        for (int d = 0; d < p->v.n; ++d) if (p->v.s0[d] % vw) return false;
        for (int d = 0; d < p->r.n; ++d) if (p->r.s0[d] % vw) return false;
        return true;
    };
    auto ok_out = [&](int vw) {
        const Radix &f = same ? p->u : p->v;
        const uint32_t tf = same ? tu : tv;
        if (out_off % vw || f.n == 0 || f.s1[0] != 1 || f.ext[0] % vw || tf % vw) return false;
        for (int d = 1; d < f.n; ++d) if (f.s1[d] % vw) return false;
        if (!same) for (int d = 0; d < p->u.n; ++d) if (p->u.s1[d] % vw) return false;
        for (int d = 0; d < p->r.n; ++d) if (p->r.s1[d] % vw) return false;
        return true;
    };
    // the transposing kernel comes in 16-byte, 8-byte (FP32) and element-wide variants, copy
    // mode in 16-byte ones through registers and 8-byte (FP32) and element-wide ones as
    // asynchronous copies into shared memory (measured: element-wise rows all in flight beat
    // 8-byte vectors through registers).  A single long run (copy mode, R empty) moves its
    // ragged tail element-wise, so only the strides matter there.
    p->single_run = (same && R.empty() && Eu > TAB) ? 1 : 0;
    const bool unit = p->u.s0[0] == 1 && p->u.s1[0] == 1 && in_off % w == 0 && out_off % w == 0;
    auto pick = [&](const auto &ok) { return ok(w) ? w : (w == 4 && ok(2)) ? 2 : 1; };
    const int vi = p->single_run ? (unit ? w : 1) : pick(ok_in);
    const int vo = p->single_run ? (unit ? w : 1) : pick(ok_out);
    const int vc = std::min(vi, vo);
    *vec_in = same ? vc : vi;
    *vec_out = same ? -vc : vo;   // negative = copy mode (no shared-memory transposition)
    if (same && !p->single_run && vc < w)   // asynchronous copy rows stage in shared memory:
        tw = std::min<uint32_t>(tw, std::max<uint32_t>(1, TILE / tu));   // keep the tile at TILE
    p->tu = tu; p->tv = tv; p->tw = tw;
    p->ll = (tu + *vec_in - 1) / *vec_in;
    p->sl = same ? 1 : (tv + vo - 1) / vo;
    p->rpp_l = 256 / p->ll;
    p->rpp_s = 256 / p->sl;
    p->fd_ll = make_fastdiv(p->ll);
    p->fd_sl = make_fastdiv(p->sl);
    p->tiles_u = (Eu + tu - 1) / tu;
    p->tiles_v = (Ev + tv - 1) / tv;
    p->tiles_w = (Er + tw - 1) / tw;
    p->fd_tiles_u = make_fastdiv(p->tiles_u);
    p->fd_tiles_v = make_fastdiv(p->tiles_v);
    p->fd_tu = make_fastdiv(tu);
    p->fd_tv = make_fastdiv(tv);
    p->fd_tuv = make_fastdiv(tu * tv);
    {   // largest input and output offsets
        int64_t mi = 0, mo = 0;
        for (int d = 0; d < n; ++d) { mi += (e2[d] - 1) * i2[d]; mo += (e2[d] - 1) * o2[d]; }
        p->off32 = (mi < (1ll << 31) - 64 && mo < (1ll << 31) - 64) ? 1 : 0;
    }
    double run_in = (double)std::min<int64_t>(pu, 64) * elem_bytes;
    double run_out = (double)std::min<int64_t>(same ? pu : pv, 64) * elem_bytes;
    *eff = run_eff(run_in) * 0.5 + run_eff(run_out) * 0.5;
}

// ------------------------------------------------------------------------------------------
// Planning
// ------------------------------------------------------------------------------------------
namespace {

struct Ctx {
    Plan *p;
    std::vector<int64_t> &ext;
    int64_t es;
};

int64_t prod_ext(const std::vector<int64_t> &ext, const std::vector<int> &labs) {
    int64_t r = 1;
    for (int l : labs) r *= ext[l];
    return r;
}

int pos_of(const std::vector<int> &v, int x) {
    for (size_t i = 0; i < v.size(); ++i) if (v[i] == x) return (int)i;
    return -1;
}

// strides (elements) of a dense column-major tensor, by label id
std::map<int, int64_t> label_strides(const std::vector<int> &labels, const std::vector<int64_t> &ext) {
    std::map<int, int64_t> s;
    int64_t st = 1;
    for (int l : labels) { s[l] = st; st *= ext[l]; }
    return s;
}

// strides of a slot as stored: the stored tensor's (views included) for inputs and the output,
// dense column-major for intermediates
std::map<int, int64_t> slot_strides(const Plan &P, const Slot &s) {
    if (s.kind == SLOT_INTER) return label_strides(s.labels, P.extent);
    return s.strides;
}

// length (elements) of the contiguous run that a group order gives in a tensor: the product of
// the leading group labels that sit at strides 1, e0, e0*e1, ... in the tensor
int64_t contiguous_run(const std::vector<int> &group, const std::map<int, int64_t> &st,
                       const std::vector<int64_t> &ext) {
    int64_t run = 1;
    for (int l : group) {
        auto it = st.find(l);
        if (it == st.end() || it->second != run) break;
        run *= ext[l];
    }
    return run;
}

void permutations(const std::vector<int> &base, std::vector<std::vector<int>> *out, size_t cap) {
    std::vector<int> v = base;
    std::sort(v.begin(), v.end());
    do {
        out->push_back(v);
        if (out->size() >= cap) break;
    } while (std::next_permutation(v.begin(), v.end()));
}

// candidate orders of one group: every permutation when few, else the orders in which the
// labels appear in the given tensors
std::vector<std::vector<int>> group_orders(const std::vector<int> &g,
                                           const std::vector<const std::vector<int> *> &tensors) {
    std::vector<std::vector<int>> res;
    if (g.size() <= 4) {
        permutations(g, &res, 24);
        return res;
    }
    for (auto *t : tensors) {
        std::vector<int> o;
        for (int l : *t) if (pos_of(g, l) >= 0) o.push_back(l);
        if (o.size() == g.size() && std::find(res.begin(), res.end(), o) == res.end()) res.push_back(o);
    }
    if (res.empty()) res.push_back(g);
    return res;
}

// modelled time of one form of a binary step
void cost_form(const Plan &P, const std::vector<int> &lx, const std::vector<int> &ly,
               const std::vector<int> &lz, bool z_free_layout, int kernel, Form *f) {
    const std::vector<int64_t> &ext = P.extent;
    double es = (double)dtype_size(P.dtype);
    const std::vector<int> &lm = f->swap ? ly : lx;   // M operand labels
    const std::vector<int> &ln = f->swap ? lx : ly;
    double M = (double)prod_ext(ext, f->M), N = (double)prod_ext(ext, f->N), K = (double)prod_ext(ext, f->K);
    auto sm = label_strides(lm, ext), sn = label_strides(ln, ext);
    std::vector<int> zl = lz;
    if (z_free_layout) { zl = f->M; zl.insert(zl.end(), f->N.begin(), f->N.end()); }
    auto sz = label_strides(zl, ext);
    double run_c = (double)contiguous_run(f->M, sz, ext);
    f->eff_store = run_eff(std::min(run_c, 32.0) * es * 2);
    double t_store = M * N * es / (kHbmBytesPerS * f->eff_store);
    if (kernel == KK_GEMM_SPLIT || kernel == KK_GEMM_EMU) {
        // pre-passes: read the operand, write 3 (split) or 6 (emulated FP64) bf16 planes in
        // [rows][K] order; the transpose engine's efficiency follows from the runs on both sides
        const bool emu = kernel == KK_GEMM_EMU;
        const double plane_bytes = emu ? 12.0 : 6.0;
        auto pre = [&](const std::vector<int> &lop, const std::vector<int> &rows, double *eff_out) {
            std::vector<int64_t> e, si, so;
            auto st = label_strides(lop, ext);
            int64_t kpad = ((int64_t)K + 7) / 8 * 8;
            int64_t s = 1;
            std::map<int, int64_t> sout;
            for (int l : f->K) { sout[l] = s; s *= ext[l]; }
            s = kpad;
            for (int l : rows) { sout[l] = s; s *= ext[l]; }
            for (int l : lop) {
                if (pos_of(f->Bt, l) >= 0) continue;   // batch labels: one pre-pass per index
                e.push_back(ext[l]); si.push_back(st[l]); so.push_back(sout[l]);
            }
            if (e.empty()) { e.push_back(1); si.push_back(1); so.push_back(1); }
            XposeParams xp;
            int vi, vo;
            double eff;
            setup_xpose((int)e.size(), e.data(), si.data(), so.data(), (int)es, &xp, &vi, &vo, &eff);
            *eff_out = eff;
            double elems = (double)prod_ext(ext, lop);
            return elems * (es + plane_bytes);
        };
        double bx = pre(lm, f->M, &f->eff_a), by = pre(ln, f->N, &f->eff_b);
        f->pre_bytes = bx + by;
        double t_pre = bx / (kHbmBytesPerS * f->eff_a) + by / (kHbmBytesPerS * f->eff_b) + 2 * kLaunchS;
        const double bn = emu ? 80.0 : 256.0, products = emu ? 21.0 : 6.0;
        double waste = (std::ceil(M / 128) * 128 * std::ceil(N / bn) * bn) / (M * N);
        double t_mma = products * 2.0 * M * N * K * waste / kBf16FlopsPerS;
        // the epilogue's stores overlap the next tile's main loop, but scattered stores still
        // cost DRAM bandwidth: charge a share of them beyond the overlap
        f->cost = t_pre + std::max(t_mma, t_store) + 0.25 * t_store + kLaunchS;
    } else {
        double ra = (double)std::max(contiguous_run(f->M, sm, ext), contiguous_run(f->K, sm, ext));
        double rb = (double)std::max(contiguous_run(f->N, sn, ext), contiguous_run(f->K, sn, ext));
        f->eff_a = run_eff(std::min(ra, 16.0) * es * 4);
        f->eff_b = run_eff(std::min(rb, 16.0) * es * 4);
        double waste = (std::ceil(M / 64) * 64 * std::ceil(N / 64) * 64) / (M * N);
        double t_mma = 2.0 * M * N * K * waste / kF64FlopsPerS;
        double t_load = (M * K / f->eff_a * std::ceil(N / 64) + N * K / f->eff_b * std::ceil(M / 64)) * es /
                        (kHbmBytesPerS * 8);   // re-reads mostly hit L2
        f->pre_bytes = 0;
        f->cost = std::max(t_mma, t_load) + t_store + kLaunchS;
    }
}

// flops of contracting the label sets of two subtrees
double step_flops(const std::vector<int64_t> &ext, const std::vector<int> &a, const std::vector<int> &b) {
    std::set<int> u(a.begin(), a.end());
    u.insert(b.begin(), b.end());
    double f = 2.0;
    for (int l : u) f *= (double)ext[l];
    return f;
}

// Pre-pass of one operand (labels in its column-major order, dense with extents ext) into
// [planes][rows][kpad] bf16 planes: K labels first (fastest), then the row group's labels.
void prepass_params(const Step &st, const std::vector<int> &labels, std::map<int, int64_t> st_,
                    int64_t in_off, const std::vector<int> &rows, const std::vector<int64_t> &ext,
                    int64_t es, XposeParams *xp, int *vec_in, int *vec_out) {
    std::map<int, int64_t> sout;
    int64_t s = 1;
    for (int l : st.form.K) { sout[l] = s; s *= ext[l]; }
    s = st.kpad;
    for (int l : rows) { sout[l] = s; s *= ext[l]; }
    std::vector<int64_t> e, a, b;
    for (int l : labels) {
        if (pos_of(st.form.Bt, l) >= 0) continue;   // one pre-pass per batch index
        e.push_back(ext[l]); a.push_back(st_[l]); b.push_back(sout[l]);
    }
    if (e.empty()) { e.push_back(1); a.push_back(1); b.push_back(1); }
    double eff;
    setup_xpose((int)e.size(), e.data(), a.data(), b.data(), (int)es, xp, vec_in, vec_out, &eff, in_off, 0);
    xp->out_plane = prod_ext(ext, rows) * st.kpad;
}

// Slices of the host-buffer pipeline (see HostPipe).  The slicing minimises a small event
// model: the inputs cross the host link one after another in the copy order, each slice's
// pre-pass runs before its first GEMM block, a block starts when its slices are pre-passed and
// the previous block is done, and results go back block by block (or column by column).  A
// GEMM takes whole waves of output tiles over the SMs, so slicing costs each block's partial
// last wave.  Candidates: equal slices, and slicings whose first slice is a half or a quarter of
// an equal one (an earlier first block) with the rest equal.
void setup_host_pipe(Plan *P, int64_t es, int want, int want_w) {
    const Step &st = P->steps[0];
    const Slot &sa = P->slots[st.a], &sb = P->slots[st.b], &sc = P->slots[st.c];
    const Slot &sm = st.form.swap ? sb : sa, &sn = st.form.swap ? sa : sb;
    HostPipe h;
    h.side = sn.elems >= sm.elems ? 1 : 0;
    const Slot &sx = h.side ? sn : sm, &sw = h.side ? sm : sn;
    const std::vector<int> &rows = h.side ? st.form.N : st.form.M;
    const std::vector<int> &wrows = h.side ? st.form.M : st.form.N;
    h.x_in = sx.index;
    h.w_in = sw.index;
    h.label = rows.back();
    h.ext = P->extent[h.label];
    if (h.ext < 2) return;
    auto tx = label_strides(sx.labels, P->extent), tc = label_strides(sc.labels, P->extent),
         tw = label_strides(sw.labels, P->extent);
    h.x_inner = tx[h.label];
    h.x_outer = sx.elems / (h.x_inner * h.ext);
    h.c_inner = tc[h.label];
    h.c_outer = sc.elems / (h.c_inner * h.ext);
    h.rows_inner = prod_ext(P->extent, rows) / h.ext;
    h.w_label = wrows.back();
    h.w_ext = P->extent[h.w_label];
    h.w_inner = tw[h.w_label];
    h.w_outer = sw.elems / (h.w_inner * h.w_ext);
    h.wc_inner = tc[h.w_label];
    h.w_rows_inner = prod_ext(P->extent, wrows) / h.w_ext;
    const bool emu = st.kernel == KK_GEMM_EMU;
    const int64_t tm = 128, tn = emu ? 80 : 256;          // output tile of the GEMM kernel
    const double prods = emu ? 21.0 / 0.6 : 6.0;             // bf16 products per tile (emu: drain-bound)
    const double t_tile = 2.0 * tm * tn * (double)st.kpad * prods / (kBf16FlopsPerS / 152);
    const double bw_in = 200e9, bw_out = 180e9, t_slice = 20e-6;
    const double planes = emu ? 12.0 : 6.0;
    const bool layout_blocks = h.wc_inner * h.w_ext == h.c_inner || h.c_inner * h.ext == h.wc_inner;
    auto tiles_of = [&](int64_t lx, int64_t lw) {
        const int64_t r = h.rows_inner * lx, rw = h.w_rows_inner * lw;
        return h.side ? ((rw + tm - 1) / tm) * ((r + tn - 1) / tn) : ((r + tm - 1) / tm) * ((rw + tn - 1) / tn);
    };
    const int64_t xu = h.x_inner * h.x_outer, wu = h.w_inner * h.w_outer;
    // slice boundaries: n slices, the first one 1/ramp of an equal slice, the rest equal (the
    // last may be shorter); empty when a slice would be empty or start off a 16-byte boundary
    auto bounds_of = [&](int64_t E, int64_t n, int64_t ramp, int64_t unit) {
        std::vector<int64_t> b;
        if (n <= 1) return std::vector<int64_t>{0, E};
        if (n > E) return b;
        const int64_t eq = (E + n - 1) / n;
        b.push_back(0);
        int64_t pos = 0;
        if (ramp > 1) {
            const int64_t first = std::max<int64_t>(1, eq / ramp);
            if (first >= eq) return std::vector<int64_t>();
            pos = first;
            b.push_back(pos);
            const int64_t c = (E - pos + (n - 1) - 1) / (n - 1);
            while (pos < E) { pos = std::min(E, pos + c); b.push_back(pos); }
        } else {
            while (pos < E) { pos = std::min(E, pos + eq); b.push_back(pos); }
        }
        for (int64_t v : b)
            if ((v * unit * es) % 16 != 0 && v != E) return std::vector<int64_t>();
        return b;
    };
    // copy order (alternating), block order (by the later of its two arrivals, then column,
    // then row), and the modelled finish time
    struct Sched { std::vector<int> copies, blocks; bool blockwise; double t; };
    auto model = [&](const std::vector<int64_t> &xb, const std::vector<int64_t> &wb) {
        Sched sd;
        const int nx = (int)xb.size() - 1, nw = (int)wb.size() - 1;
        sd.blockwise = layout_blocks && (nx > 1 || nw > 1);
        std::vector<int> posx(nx), posw(nw);
        for (int k = 0; k < std::max(nx, nw); ++k) {
            if (k < nw) { posw[k] = (int)sd.copies.size(); sd.copies.push_back(-1 - k); }
            if (k < nx) { posx[k] = (int)sd.copies.size(); sd.copies.push_back(k); }
        }
        auto lx = [&](int j) { return xb[j + 1] - xb[j]; };
        auto lw = [&](int i) { return wb[i + 1] - wb[i]; };
        auto xbytes = [&](int j) { return (double)h.x_inner * lx(j) * h.x_outer * es; };
        auto cbytes = [&](int j) { return (double)h.c_inner * lx(j) * h.c_outer * es; };
        auto wbytes = [&](int i) { return (double)h.w_inner * lw(i) * h.w_outer * es; };
        std::vector<double> rx(nx), rw(nw);
        double c = 0;
        for (int q : sd.copies) {
            if (q >= 0) { c += (xbytes(q) + (P->op != 0 ? cbytes(q) : 0)) / bw_in; rx[q] = c; }
            else { c += wbytes(-1 - q) / bw_in; rw[-1 - q] = c; }
        }
        for (int i = 0; i < nw; ++i)
            for (int j = 0; j < nx; ++j) sd.blocks.push_back(i * nx + j);
        std::stable_sort(sd.blocks.begin(), sd.blocks.end(), [&](int u, int v) {
            const int iu = u / nx, ju = u % nx, iv = v / nx, jv = v % nx;
            const int au = std::max(posw[iu], posx[ju]), av = std::max(posw[iv], posx[jv]);
            if (au != av) return au < av;
            if (ju != jv) return ju < jv;
            return iu < iv;
        });
        const bool sliced = nx > 1 || nw > 1;
        std::vector<char> px(nx, 0), pw(nw, 0);
        std::vector<int> left(nx, nw);
        double t = 0, out = 0;
        for (int u : sd.blocks) {
            const int i = u / nx, j = u % nx;
            if (!pw[i]) { t = std::max(t, rw[i]) + wbytes(i) / es * (es + planes) / kHbmBytesPerS; pw[i] = 1; }
            if (!px[j]) { t = std::max(t, rx[j]) + xbytes(j) / es * (es + planes) / kHbmBytesPerS; px[j] = 1; }
            t += (double)((tiles_of(lx(j), lw(i)) + 151) / 152) * t_tile + (sliced ? t_slice : 0);
            if (sd.blockwise) out = std::max(out, t) + cbytes(j) * (double)lw(i) / (double)h.w_ext / bw_out;
            else if (--left[j] == 0) out = std::max(out, t) + cbytes(j) / bw_out;
        }
        sd.t = std::max(out, t);
        return sd;
    };
    const std::vector<int64_t> one_x = {0, h.ext}, one_w = {0, h.w_ext};
    Sched best = model(one_x, one_w);
    std::vector<int64_t> bx = one_x, bw = one_w;
    h.model_s[0] = best.t;
    const bool forced = want > 1 || want_w > 1;
    std::vector<std::vector<int64_t>> cand_x, cand_w;
    if (want > 1) cand_x.push_back(bounds_of(h.ext, std::min<int64_t>(want, h.ext), 1, xu));
    else for (int n : {1, 2, 3, 4, 6, 8}) for (int r : {1, 2, 4}) if (n > 1 || r == 1) cand_x.push_back(bounds_of(h.ext, n, r, xu));
    if (want_w > 1) cand_w.push_back(bounds_of(h.w_ext, std::min<int64_t>(want_w, h.w_ext), 1, wu));
    else if (want_w == 0) { for (int n : {1, 2, 3, 4, 6, 8}) for (int r : {1, 2, 4}) if (n > 1 || r == 1) cand_w.push_back(bounds_of(h.w_ext, n, r, wu)); }
    else cand_w.push_back(one_w);
    // among the candidates the model finishes within 1 % of the first one, the one with the
    // fewest GEMM blocks (the model does not see every cost of a small block); unless forced,
    // it must beat no slicing by 3 %
    struct Cand { Sched sd; std::vector<int64_t> xb, wb; };
    std::vector<Cand> cands;
    const double t_whole = best.t;
    for (const auto &xb : cand_x)
        for (const auto &wb : cand_w) {
            if (xb.size() < 2 || wb.size() < 2) continue;
            const int nx = (int)xb.size() - 1, nw = (int)wb.size() - 1;
            if ((nx == 1 && nw == 1) || nx + nw > 31 || nx * nw > 64) continue;
            cands.push_back(Cand{model(xb, wb), xb, wb});
        }
    if (cands.empty()) return;
    double t_min = cands[0].sd.t;
    for (const Cand &c : cands) t_min = std::min(t_min, c.sd.t);
    const Cand *pick = nullptr;
    for (const Cand &c : cands) {
        if (c.sd.t > t_min * 1.01) continue;
        if (!pick || c.sd.blocks.size() < pick->sd.blocks.size() ||
            (c.sd.blocks.size() == pick->sd.blocks.size() && c.sd.t < pick->sd.t))
            pick = &c;
    }
    if (!forced && pick->sd.t > t_whole * 0.97) return;
    best = pick->sd;
    bx = pick->xb;
    bw = pick->wb;
    h.xb = bx;
    h.wb = bw;
    h.n_chunks = (int)bx.size() - 1;
    h.w_n = (int)bw.size() - 1;
    h.copies = best.copies;
    h.blocks = best.blocks;
    h.blockwise = best.blockwise;
    h.model_s[1] = best.t;
    h.pre.resize(h.n_chunks);
    h.pre_vec.assign(h.n_chunks, 1);
    h.pre_vout.assign(h.n_chunks, 1);
    for (int j = 0; j < h.n_chunks; ++j) {
        std::vector<int64_t> e = P->extent;
        e[h.label] = bx[j + 1] - bx[j];
        prepass_params(st, sx.labels, label_strides(sx.labels, e), 0, rows, e, es, &h.pre[j], &h.pre_vec[j],
                       &h.pre_vout[j]);
    }
    h.w_pre.resize(h.w_n);
    h.w_pre_vec.assign(h.w_n, 1);
    h.w_pre_vout.assign(h.w_n, 1);
    for (int i = 0; i < h.w_n; ++i) {
        std::vector<int64_t> ew = P->extent;
        ew[h.w_label] = bw[i + 1] - bw[i];
        prepass_params(st, sw.labels, label_strides(sw.labels, ew), 0, wrows, ew, es, &h.w_pre[i], &h.w_pre_vec[i],
                       &h.w_pre_vout[i]);
    }
    h.ok = true;
    P->pipe = h;
}

}  // namespace

comet_status_t build_plan(const char *expr, const comet_extent_t *extents, int n_extents,
                          const comet_view_t *views, int n_views, const comet_dtype_t *dtypes,
                          int n_dtypes, const comet_plan_opts_t *opts_in, Plan *P, std::string *err) {
    if (!expr) return COMET_ERR_NULL;
    comet_plan_opts_t opts;
    comet_plan_opts_default(&opts);
    if (opts_in) opts = *opts_in;
    if (opts.precision != COMET_PREC_NATIVE && opts.precision != COMET_PREC_SPLIT_BF16 &&
        opts.precision != COMET_PREC_EMU_F64) {
        *err = "unknown precision"; return COMET_ERR_ARG;
    }
    if (opts.kc < 0 || opts.timeout_ms < 0) { *err = "negative kc or timeout"; return COMET_ERR_ARG; }
    P->opts = opts;
    P->expr = expr;
    comet_status_t st = parse_expr(expr, &P->parsed, err);
    if (st != COMET_OK) return st;
    const ParsedExpr &E = P->parsed;
    P->n_in = (int)E.ins.size();
    P->op = E.op;
    P->alpha = E.alpha * opts.alpha;
    // labels: ids in order of first appearance on the right-hand side
    std::map<std::string, int> id;
    for (auto &t : E.ins)
        for (auto &l : t.labels)
            if (!id.count(l)) { id[l] = (int)P->label_names.size(); P->label_names.push_back(l); }
    for (auto &l : E.out.labels)
        if (!id.count(l)) { *err = "output label " + l + " is on no right-hand operand"; return COMET_ERR_LABEL; }
    int L = (int)P->label_names.size();
    if (L > 64) { *err = "too many labels"; return COMET_ERR_UNSUPPORTED; }
    P->extent.assign(L, -1);
    if (n_extents < 0 || (n_extents > 0 && !extents)) return COMET_ERR_NULL;
    for (int i = 0; i < n_extents; ++i) {
        if (!extents[i].label) return COMET_ERR_NULL;
        auto it = id.find(extents[i].label);
        if (it == id.end()) continue;   // extents for unused labels are ignored
        if (extents[i].extent <= 0) { *err = std::string("non-positive extent for ") + extents[i].label; return COMET_ERR_SHAPE; }
        if (P->extent[it->second] != -1 && P->extent[it->second] != extents[i].extent) {
            *err = std::string("two extents for ") + extents[i].label; return COMET_ERR_SHAPE;
        }
        P->extent[it->second] = extents[i].extent;
    }
    for (int l = 0; l < L; ++l)
        if (P->extent[l] < 0) { *err = "no extent for label " + P->label_names[l]; return COMET_ERR_LABEL; }
    // dtypes
    if (!dtypes) return COMET_ERR_NULL;
    if (n_dtypes != P->n_in + 1) { *err = "one dtype per operand and one for the output"; return COMET_ERR_DTYPE; }
    for (int i = 0; i < n_dtypes; ++i) {
        if (dtypes[i] != COMET_F32 && dtypes[i] != COMET_F64) { *err = "unknown dtype"; return COMET_ERR_DTYPE; }
        if (dtypes[i] != dtypes[0]) { *err = "operands of different dtypes"; return COMET_ERR_DTYPE; }
    }
    P->dtype = dtypes[0];
    if (opts.precision == COMET_PREC_EMU_F64 && P->dtype != COMET_F64) {
        *err = "the emulated FP64 precision takes FP64 operands"; return COMET_ERR_DTYPE;
    }
    // labelled tensors as id lists (each label once; a label written twice is a diagonal);
    // structural checks (Section 2: contraction vs free labels)
    std::vector<std::vector<int>> written;   // per tensor (inputs, then the output): labels as written
    for (auto &t : E.ins) {
        std::vector<int> v;
        for (auto &l : t.labels) v.push_back(id[l]);
        if (v.size() > (size_t)kMaxRank) { *err = "rank above 8"; return COMET_ERR_UNSUPPORTED; }
        written.push_back(v);
    }
    {
        std::vector<int> v;
        for (auto &l : E.out.labels) v.push_back(id[l]);
        if (v.size() > (size_t)kMaxRank) { *err = "rank above 8"; return COMET_ERR_UNSUPPORTED; }
        written.push_back(v);
    }
    auto unique_of = [&](const std::vector<int> &v) {
        std::vector<int> u;
        for (int l : v) if (pos_of(u, l) < 0) u.push_back(l);
        return u;
    };
    std::vector<std::vector<int>> in_labs;
    for (int t = 0; t < P->n_in; ++t) in_labs.push_back(unique_of(written[t]));
    std::vector<int> out_labs = unique_of(written[P->n_in]);
    // views: per written dimension (declared extent, lo, step); default the whole dimension
    const int n_t = P->n_in + 1;
    std::vector<std::vector<int64_t>> decl(n_t), lo(n_t), step(n_t);
    for (int t = 0; t < n_t; ++t)
        for (int l : written[t]) { decl[t].push_back(P->extent[l]); lo[t].push_back(0); step[t].push_back(1); }
    if (n_views < 0 || (n_views > 0 && !views)) return COMET_ERR_NULL;
    {
        std::set<std::pair<int, int>> seen;
        for (int v = 0; v < n_views; ++v) {
            const comet_view_t &w = views[v];
            if (w.operand < 0 || w.operand >= n_t || w.dim < 0 || w.dim >= (int)written[w.operand].size()) {
                *err = "view: operand or dimension out of range"; return COMET_ERR_ARG;
            }
            if (!seen.insert({w.operand, w.dim}).second) { *err = "view: dimension given twice"; return COMET_ERR_ARG; }
            const int64_t n = P->extent[written[w.operand][w.dim]];
            if (w.declared < 1 || w.lo < 0 || w.step < 1 ||
                (long double)w.lo + (long double)(n - 1) * (long double)w.step >= (long double)w.declared) {
                *err = "view: range outside the declared extent"; return COMET_ERR_SHAPE;
            }
            decl[w.operand][w.dim] = w.declared;
            lo[w.operand][w.dim] = w.lo;
            step[w.operand][w.dim] = w.step;
        }
    }
    std::vector<int> count(L, 0);
    for (auto &v : in_labs) for (int l : v) ++count[l];
    for (int l : out_labs) ++count[l];
    // labels on a single operand and not on the output are summed inside that operand first
    // (a reduction step); the rest of the plan sees the reduced operand
    if (E.has_sum) {
        std::set<std::string> want, got(E.sum_labels.begin(), E.sum_labels.end());
        for (int l = 0; l < L; ++l) if (pos_of(out_labs, l) < 0) want.insert(P->label_names[l]);
        if (want != got) { *err = "sum_{...} does not name the summed labels"; return COMET_ERR_LABEL; }
    }
    // sizes
    auto elems_of = [&](const std::vector<int> &v) {
        long double e = 1;
        for (int l : v) e *= (long double)P->extent[l];
        return e;
    };
    for (auto &v : in_labs) if (elems_of(v) > 9.0e15L) { *err = "tensor too large"; return COMET_ERR_SHAPE; }
    if (elems_of(out_labs) > 9.0e15L) { *err = "tensor too large"; return COMET_ERR_SHAPE; }
    size_t es = dtype_size(P->dtype);

    // slots: inputs, then the output, with the strides of their stored tensors
    auto stored_layout = [&](int t, Slot *s) -> comet_status_t {
        long double storage = 1;
        int64_t S = 1;
        s->offset = 0;
        s->strides.clear();
        for (size_t d = 0; d < written[t].size(); ++d) {
            s->strides[written[t][d]] += step[t][d] * S;
            s->offset += lo[t][d] * S;
            storage *= (long double)decl[t][d];
            if (storage > 9.0e15L) { *err = "tensor too large"; return COMET_ERR_SHAPE; }
            S *= decl[t][d];
        }
        s->storage = (int64_t)storage;
        // declared >= lo + (n-1) step + 1 >= n: with no repeated label, offset 0 and
        // storage = elems, every dimension is whole (dense)
        s->view = written[t].size() != s->labels.size() || s->offset != 0 || s->storage != s->elems;
        if (s->view) {
            if (s->elems >= (1ll << 31)) { *err = "views of 2^31 elements or more"; return COMET_ERR_UNSUPPORTED; }
            std::vector<int> byst = s->labels;   // abs-max walk: smallest stride first
            std::stable_sort(byst.begin(), byst.end(), [&](int a, int b) { return s->strides[a] < s->strides[b]; });
            std::vector<int64_t> ex(P->extent.begin(), P->extent.end()), s0(P->extent.size(), 0),
                s1(P->extent.size(), 0);
            for (int l : byst) s0[l] = s->strides[l];
            fill_radix(&s->vradix, byst, ex.data(), s0.data(), s1.data());
            s->vradix.total = (uint32_t)s->elems;
        }
        return COMET_OK;
    };
    for (int i = 0; i < P->n_in; ++i) {
        Slot s; s.kind = SLOT_INPUT; s.index = i; s.labels = in_labs[i];
        s.elems = (int64_t)elems_of(in_labs[i]);
        comet_status_t vs = stored_layout(i, &s);
        if (vs != COMET_OK) return vs;
        P->slots.push_back(s);
    }
    Slot so; so.kind = SLOT_OUTPUT; so.labels = out_labs; so.elems = (int64_t)elems_of(out_labs);
    {
        comet_status_t vs = stored_layout(P->n_in, &so);
        if (vs != COMET_OK) return vs;
    }
    int out_slot = (int)P->slots.size();
    P->slots.push_back(so);

    // ---- reductions of labels private to one operand ----
    std::vector<int> leaf_slot(P->n_in);
    for (int t = 0; t < P->n_in; ++t) {
        leaf_slot[t] = t;
        std::vector<int> keep;
        for (int l : in_labs[t]) if (count[l] > 1) keep.push_back(l);
        if (keep.size() == in_labs[t].size()) continue;
        Step r;
        r.kernel = KK_REDUCE;
        r.a = t;
        r.flops = (double)elems_of(in_labs[t]);
        if (P->n_in == 1) {
            r.c = out_slot;
            r.final_step = true;
        } else {
            Slot s; s.kind = SLOT_INTER; s.labels = keep; s.elems = (int64_t)elems_of(keep);
            r.c = (int)P->slots.size();
            P->slots.push_back(s);
            leaf_slot[t] = r.c;
        }
        P->steps.push_back(r);
        in_labs[t] = keep;
    }
    // ---- single operand: scaled copy / transpose (ta.copy), or the reduction above ----
    if (P->n_in == 1) {
        if (P->steps.empty()) {
            Step s; s.a = 0; s.c = out_slot; s.kernel = KK_COPY; s.final_step = true; s.flops = 0;
            P->steps.push_back(s);
        }
        P->tree = E.ins[0].name;
    } else {
        // ---- operand order (Section 6): DP over subsets, min flops; ties: min intermediate
        // elements, then the left-most split ----
        int n = P->n_in;
        if (n > 12) { *err = "more than 12 operands"; return COMET_ERR_UNSUPPORTED; }
        int full = (1 << n) - 1;
        // labels of the intermediate of subset S: labels of S that also occur outside S
        std::vector<std::vector<int>> sub_labels(1 << n);
        for (int S = 1; S <= full; ++S) {
            std::vector<int> inside(L, 0), outside(L, 0);
            for (int t = 0; t < n; ++t)
                for (int l : in_labs[t]) { if (S >> t & 1) inside[l] = 1; else outside[l] = 1; }
            for (int l : out_labs) outside[l] = 1;
            for (int l = 0; l < L; ++l) if (inside[l] && outside[l]) sub_labels[S].push_back(l);
        }
        const double INF = std::numeric_limits<double>::infinity();
        std::vector<double> best_f(1 << n, INF), best_b(1 << n, INF);
        std::vector<int> split(1 << n, 0);
        for (int t = 0; t < n; ++t) { best_f[1 << t] = 0; best_b[1 << t] = 0; }
        auto inter_bytes = [&](int S) { return (double)elems_of(sub_labels[S]) * es; };
        auto natural_split = [&](int S) {   // left-to-right: split off the highest operand
            int hi = 31 - __builtin_clz((unsigned)S);
            return S & ~(1 << hi);
        };
        for (int S = 1; S <= full; ++S) {
            if (__builtin_popcount((unsigned)S) < 2) continue;
            if (opts.order == COMET_ORDER_NATURAL) {
                int Lp = natural_split(S), R = S ^ Lp;
                split[S] = Lp;
                best_f[S] = best_f[Lp] + best_f[R] + step_flops(P->extent, sub_labels[Lp], sub_labels[R]);
                best_b[S] = best_b[Lp] + best_b[R] + (S == full ? 0 : inter_bytes(S));
                continue;
            }
            // enumerate L as a proper subset containing the lowest operand of S (each split once)
            int low = S & -S;
            for (int Lp = (S - 1) & S; Lp > 0; Lp = (Lp - 1) & S) {
                if (!(Lp & low)) continue;
                int R = S ^ Lp;
                if (best_f[Lp] == INF || best_f[R] == INF) continue;
                double ib = (S == full) ? 0 : inter_bytes(S);
                if (S != full && opts.workspace_cap && ib > (double)opts.workspace_cap) continue;
                double f = best_f[Lp] + best_f[R] + step_flops(P->extent, sub_labels[Lp], sub_labels[R]);
                double b = best_b[Lp] + best_b[R] + ib;
                // ties: fewer flops, fewer intermediate bytes, then the smaller (left-most) split
                bool better = f < best_f[S] * (1 - 1e-12) ||
                              (std::fabs(f - best_f[S]) <= 1e-12 * f &&
                               (b < best_b[S] || (b == best_b[S] && Lp < split[S])));
                if (better || best_f[S] == INF) { best_f[S] = f; best_b[S] = b; split[S] = Lp; }
            }
        }
        if (best_f[full] == INF) { *err = "no order fits the workspace cap"; return COMET_ERR_WORKSPACE; }
        P->flops = best_f[full];
        // natural order flops for reference
        {
            double f = 0;
            int S = 1;
            for (int t = 1; t < n; ++t) {
                int R = 1 << t;
                f += step_flops(P->extent, sub_labels[S], sub_labels[R]);
                S |= R;
            }
            P->flops_natural = f;
        }
        // emit steps post-order
        std::function<int(int)> emit = [&](int S) -> int {
            if (__builtin_popcount((unsigned)S) == 1) return leaf_slot[__builtin_ctz((unsigned)S)];
            int Lp = split[S], R = S ^ Lp;
            int a = emit(Lp), b = emit(R);
            int c;
            if (S == full) {
                c = out_slot;
            } else {
                Slot s; s.kind = SLOT_INTER; s.labels = sub_labels[S];
                s.elems = (int64_t)elems_of(sub_labels[S]);
                c = (int)P->slots.size();
                P->slots.push_back(s);
            }
            Step st; st.a = a; st.b = b; st.c = c; st.final_step = (S == full);
            st.flops = step_flops(P->extent, sub_labels[Lp], sub_labels[R]);
            P->steps.push_back(st);
            return c;
        };
        std::function<std::string(int)> tree = [&](int S) -> std::string {
            if (__builtin_popcount((unsigned)S) == 1) return E.ins[__builtin_ctz((unsigned)S)].name;
            return "(" + tree(split[S]) + "*" + tree(S ^ split[S]) + ")";
        };
        emit(full);
        P->tree = tree(full);
    }

    // ---- TTGT form of every binary step (Section 6) ----
    int kernel = opts.precision == COMET_PREC_SPLIT_BF16 ? KK_GEMM_SPLIT
                 : opts.precision == COMET_PREC_EMU_F64 ? KK_GEMM_EMU : KK_GEMM_F64;
    for (auto &st : P->steps) {
        if (st.kernel == KK_COPY || st.kernel == KK_REDUCE) continue;
        st.kernel = kernel;
        Slot &sa = P->slots[st.a], &sb = P->slots[st.b], &sc = P->slots[st.c];
        bool free_layout = sc.kind == SLOT_INTER;
        // free in a, free in b, contracted, batch (on both inputs and kept in the result)
        std::vector<int> I, J, K, Bt;
        for (int l : sa.labels) {
            if (pos_of(sb.labels, l) < 0) I.push_back(l);
            else (pos_of(sc.labels, l) >= 0 ? Bt : K).push_back(l);
        }
        for (int l : sb.labels) if (pos_of(sa.labels, l) < 0) J.push_back(l);
        for (int l : sc.labels)
            if (pos_of(I, l) < 0 && pos_of(J, l) < 0 && pos_of(Bt, l) < 0) {
                *err = "internal: output label not free"; return COMET_ERR_INTERNAL;
            }
        if (prod_ext(P->extent, I) >= (1ll << 31) || prod_ext(P->extent, J) >= (1ll << 31) ||
            prod_ext(P->extent, K) >= (1ll << 31)) {
            *err = "a merged GEMM dimension reaches 2^31"; return COMET_ERR_UNSUPPORTED;
        }
        if (kernel == KK_GEMM_EMU && prod_ext(P->extent, K) > 98304) {
            *err = "the emulated FP64 precision takes a merged contraction length of at most 98304";
            return COMET_ERR_UNSUPPORTED;
        }
        std::vector<Form> forms;
        for (int swap = 0; swap < 2; ++swap) {
            const std::vector<int> &gm = swap ? J : I, &gn = swap ? I : J;
            const std::vector<int> &lm = swap ? sb.labels : sa.labels, &ln = swap ? sa.labels : sb.labels;
            auto om = group_orders(gm, {&sc.labels, &lm});
            auto on = group_orders(gn, {&sc.labels, &ln});
            auto ok = group_orders(K, {&lm, &ln});
            for (auto &m : om) for (auto &nn : on) for (auto &k : ok) {
                Form f; f.swap = swap; f.M = m; f.N = nn; f.K = k; f.Bt = Bt;
                cost_form(*P, sa.labels, sb.labels, sc.labels, free_layout, kernel, &f);
                forms.push_back(f);
                if (forms.size() > 20000) break;
            }
        }
        st.n_forms = (int)forms.size();
        int pick = 0;
        if (opts.form >= 0) {
            pick = opts.form % st.n_forms;
        } else {
            for (int i = 1; i < st.n_forms; ++i)
                if (forms[i].cost < forms[pick].cost * (1 - 1e-9)) pick = i;
        }
        st.form = forms[pick];
        st.form_index = pick;
        // one operand without free labels: a tensor-times-vector step (HBM-bound, see k_gemv.cu)
        if (st.form.M.empty() || st.form.N.empty()) st.kernel = KK_GEMV;
        if (free_layout) {   // the intermediate is stored as [M][N][batch]: the epilogue writes rows
            sc.labels = st.form.M;
            sc.labels.insert(sc.labels.end(), st.form.N.begin(), st.form.N.end());
            sc.labels.insert(sc.labels.end(), st.form.Bt.begin(), st.form.Bt.end());
        }
        if (prod_ext(P->extent, Bt) >= (1ll << 31)) { *err = "batch labels reach 2^31 indices"; return COMET_ERR_UNSUPPORTED; }
        {   // batch offsets of the three tensors (strides of their full layouts)
            auto ta = slot_strides(*P, sa), tb = slot_strides(*P, sb), tc = slot_strides(*P, sc);
            st.n_batch = 1;
            for (int l : Bt) {
                st.bt_ext.push_back(P->extent[l]);
                st.bt_sa.push_back(ta[l]);
                st.bt_sb.push_back(tb[l]);
                st.bt_sc.push_back(tc[l]);
                st.n_batch *= P->extent[l];
            }
        }
    }

    // ---- workspace: intermediates, then one region for the split parts of any step ----
    size_t off = 0;
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    for (auto &s : P->slots)
        if (s.kind == SLOT_INTER) { s.ws_off = off; off = align(off + (size_t)s.elems * es); }
    size_t parts_base = off, parts_max = 0;
    for (auto &st : P->steps) {
        if (st.kernel != KK_GEMM_SPLIT && st.kernel != KK_GEMM_EMU) continue;
        int64_t Kx = prod_ext(P->extent, st.form.K);
        st.kpad = (Kx + 7) / 8 * 8;
        int64_t rows_a = prod_ext(P->extent, st.form.M), rows_b = prod_ext(P->extent, st.form.N);
        const size_t planes = st.kernel == KK_GEMM_EMU ? 6 : 3;
        size_t ba = align(planes * rows_a * st.kpad * 2), bb = align(planes * rows_b * st.kpad * 2);
        st.ws_parts_a = parts_base;
        st.ws_parts_b = parts_base + ba;
        // K slices: a split GEMM with fewer output tiles than SMs spreads K over more work items
        // (slices of at least 256 K values, partials at most 256 MB)
        st.ksplit = 1;
        if (st.kernel == KK_GEMM_SPLIT && opts.ksplit != 1) {
            const int64_t tiles = ((rows_a + 127) / 128) * ((rows_b + 255) / 256);
            const int64_t nkb = (Kx + 31) / 32;
            int64_t k = opts.ksplit > 1 ? opts.ksplit
                                        : std::min<int64_t>({(152 + tiles - 1) / tiles, nkb / 8, 16});
            while (k > 1 && (double)k * tiles * 128 * 256 * 4 > 256.0 * (1 << 20)) --k;
            st.ksplit = (uint32_t)std::max<int64_t>(1, std::min<int64_t>(k, nkb));
        }
        st.ws_ksplit = parts_base + ba + bb;
        // partials: every tile's K slices (128 x 256 floats per tile and slice), or with whole-K
        // tiles the slices of a partial last wave over 152 SMs (at most 152 tile slices)
        const int64_t tiles = ((rows_a + 127) / 128) * ((rows_b + 255) / 256);
        size_t bk = 0;
        if (st.ksplit > 1) bk = (size_t)st.ksplit * tiles * 128 * 256 * 4;
        else if (st.kernel == KK_GEMM_SPLIT && tiles > 152) bk = (size_t)152 * 128 * 256 * 4;
        // the launch's tail rule on a 152-SM GB300 (it applies the rule to the device's own count)
        st.tail_tiles = 0;
        st.tail_slices = 1;
        if (st.kernel == KK_GEMM_SPLIT && st.ksplit == 1 && tiles > 152 && tiles % 152 != 0 &&
            2 * (tiles % 152) <= 152) {
            st.tail_tiles = (uint32_t)(tiles % 152);
            st.tail_slices = (uint32_t)std::min<int64_t>({4, 152 / (tiles % 152), (Kx + 31) / 32});
        }
        st.ksplit_bytes = bk;
        parts_max = std::max(parts_max, ba + bb + align(bk));
    }
    for (auto &st : P->steps) {
        if (st.kernel == KK_REDUCE) {   // y[kept] = sum over the private labels of the operand
            const Slot &sa = P->slots[st.a], &sc = P->slots[st.c];
            auto ta = slot_strides(*P, sa), tc = slot_strides(*P, sc);
            std::vector<int> kept = sc.labels, summed;
            for (int l : sa.labels) if (pos_of(kept, l) < 0) summed.push_back(l);
            std::vector<int64_t> ex(P->extent.begin(), P->extent.end()), s0(L, 0), s1(L, 0), zero(L, 0);
            GemvParams &v = st.gemv;
            std::memset(&v, 0, sizeof(v));
            for (int l : kept) { s0[l] = ta[l]; s1[l] = tc[l]; }
            fill_radix(&v.n, kept, ex.data(), s0.data(), s1.data());
            for (int l : summed) { s0[l] = 0; s1[l] = ta[l]; }
            fill_radix(&v.k, summed, ex.data(), s0.data(), s1.data());
            v.N = (uint32_t)prod_ext(P->extent, kept);
            v.K = (uint32_t)prod_ext(P->extent, summed);
            v.n.total = v.N;
            v.k.total = v.K;
            if (prod_ext(P->extent, kept) >= (1ll << 31) || prod_ext(P->extent, summed) >= (1ll << 31)) {
                *err = "a reduction dimension reaches 2^31"; return COMET_ERR_UNSUPPORTED;
            }
            int64_t min_n = INT64_MAX, min_k = INT64_MAX;
            for (int d = 0; d < v.n.n; ++d) min_n = std::min(min_n, v.n.s0[d]);
            for (int d = 0; d < v.k.n; ++d) min_k = std::min(min_k, v.k.s1[d]);
            v.n_fast = min_n < min_k ? 1 : 0;
            v.nchunks = (v.K + 1023) / 1024;
            v.v_ones = 1;
            v.n_batch = 1;
            v.bv.total = 1;
            v.by.total = 1;
            st.ws_partial = parts_base;
            parts_max = std::max(parts_max, align((size_t)v.nchunks * (size_t)v.N * 8));
            continue;
        }
        if (st.kernel != KK_GEMV) continue;
        const int64_t Kx = prod_ext(P->extent, st.form.K);
        const int64_t Nx = prod_ext(P->extent, st.form.M.empty() ? st.form.N : st.form.M);
        st.ws_partial = parts_base;
        parts_max = std::max(parts_max, align((size_t)st.n_batch * (size_t)((Kx + 1023) / 1024) * (size_t)Nx * 8));
    }
    bool any_split = false;
    for (auto &st : P->steps) any_split |= st.kernel == KK_GEMM_SPLIT || st.kernel == KK_GEMM_EMU;
    for (auto &st : P->steps) st.ws_scales = parts_base + parts_max;
    P->workspace = parts_base + parts_max + (any_split ? 256 : 0);

    // ---- precomputed parameter blocks ----
    for (auto &st : P->steps) {
        if (st.kernel == KK_REDUCE) continue;
        if (st.kernel == KK_COPY) {
            const Slot &sa = P->slots[st.a], &sc = P->slots[st.c];
            auto si = slot_strides(*P, sa), so2 = slot_strides(*P, sc);
            std::vector<int64_t> e, a, b;
            for (int l : sa.labels) { e.push_back(P->extent[l]); a.push_back(si[l]); b.push_back(so2[l]); }
            double eff;
            setup_xpose((int)e.size(), e.data(), a.data(), b.data(), (int)es, &st.copy,
                        &st.copy_vec_in, &st.copy_vec_out, &eff, sa.kind == SLOT_INTER ? 0 : sa.offset,
                        sc.kind == SLOT_INTER ? 0 : sc.offset);
            continue;
        }
        const Slot &sa = P->slots[st.a], &sb = P->slots[st.b], &sc = P->slots[st.c];
        const Slot &sm = st.form.swap ? sb : sa, &sn = st.form.swap ? sa : sb;
        auto tm = slot_strides(*P, sm), tn = slot_strides(*P, sn), tc = slot_strides(*P, sc);
        GemmParams &g = st.gemm;
        std::memset(&g, 0, sizeof(g));
        std::vector<int64_t> ex(P->extent.begin(), P->extent.end());
        std::vector<int64_t> s0(L), s1(L);
        // M: (A strides, C strides)
        for (int l : st.form.M) { s0[l] = tm[l]; s1[l] = tc[l]; }
        fill_radix(&g.ma, st.form.M, ex.data(), s0.data(), s1.data());
        for (int l : st.form.N) { s0[l] = tn[l]; s1[l] = tc[l]; }
        fill_radix(&g.nb, st.form.N, ex.data(), s0.data(), s1.data());
        for (int l : st.form.K) { s0[l] = tm[l]; s1[l] = tn[l]; }
        fill_radix(&g.k, st.form.K, ex.data(), s0.data(), s1.data());
        g.M = (uint32_t)prod_ext(P->extent, st.form.M);
        g.N = (uint32_t)prod_ext(P->extent, st.form.N);
        g.K = (uint32_t)prod_ext(P->extent, st.form.K);
        g.ma.total = g.M; g.nb.total = g.N; g.k.total = g.K;
        if (st.kernel == KK_GEMV) {
            GemvParams &v = st.gemv;
            std::memset(&v, 0, sizeof(v));
            st.gemv_vec_is_a = st.form.M.empty();
            if (st.gemv_vec_is_a) {          // y[n] = sum_k A[k] B[k, n]
                v.n = g.nb;
                v.k = g.k;
                v.N = g.N;
            } else {                         // y[m] = sum_k A[m, k] B[k]
                v.n = g.ma;
                v.k = g.k;
                for (int d = 0; d < v.k.n; ++d) std::swap(v.k.s0[d], v.k.s1[d]);
                v.N = g.M;
            }
            v.K = g.K;
            v.n.total = v.N;
            v.k.total = v.K;
            int64_t min_n = INT64_MAX, min_k = INT64_MAX;
            for (int d = 0; d < v.n.n; ++d) min_n = std::min(min_n, v.n.s0[d]);
            for (int d = 0; d < v.k.n; ++d) min_k = std::min(min_k, v.k.s1[d]);
            v.n_fast = min_n < min_k ? 1 : 0;
            v.nchunks = (v.K + 1023) / 1024;
            {   // batch digits in-kernel: (vector, large operand) offsets and result offsets
                std::vector<int> none;
                std::vector<int64_t> sv(L, 0), sx(L, 0), sy(L, 0), zero(L, 0);
                auto ta = slot_strides(*P, sa), tb = slot_strides(*P, sb), tc = slot_strides(*P, sc);
                for (int l : st.form.Bt) {
                    sv[l] = st.gemv_vec_is_a ? (st.form.swap ? tb[l] : ta[l]) : (st.form.swap ? ta[l] : tb[l]);
                    sx[l] = st.gemv_vec_is_a ? (st.form.swap ? ta[l] : tb[l]) : (st.form.swap ? tb[l] : ta[l]);
                    sy[l] = tc[l];
                }
                fill_radix(&v.bv, st.form.Bt, ex.data(), sv.data(), sx.data());
                fill_radix(&v.by, st.form.Bt, ex.data(), sy.data(), zero.data());
                v.n_batch = (uint32_t)st.n_batch;
            }
            continue;
        }
        if (st.kernel == KK_GEMM_SPLIT || st.kernel == KK_GEMM_EMU) {
            // pre-pass of each operand into [planes][rows][kpad] bf16 planes (K order, then rows)
            prepass_params(st, sm.labels, slot_strides(*P, sm), sm.kind == SLOT_INTER ? 0 : sm.offset,
                           st.form.M, P->extent, es, &st.pre_a, &st.pre_a_vec, &st.pre_a_vout);
            prepass_params(st, sn.labels, slot_strides(*P, sn), sn.kind == SLOT_INTER ? 0 : sn.offset,
                           st.form.N, P->extent, es, &st.pre_b, &st.pre_b_vec, &st.pre_b_vout);
        }
    }
    // ---- host-buffer pipeline of one-step split / emulated plans (comet_contract_host) ----
    P->pipe = HostPipe();
    if (P->steps.size() == 1 && opts.host_slices != 1) {
        const Step &st = P->steps[0];
        if ((st.kernel == KK_GEMM_SPLIT || st.kernel == KK_GEMM_EMU) && st.n_batch == 1 && st.b >= 0 && P->slots[st.a].kind == SLOT_INPUT &&
            P->slots[st.b].kind == SLOT_INPUT && P->slots[st.c].kind == SLOT_OUTPUT &&
            !st.form.M.empty() && !st.form.N.empty() && !P->slots[st.a].view &&
            !P->slots[st.b].view && !P->slots[st.c].view)
            setup_host_pipe(P, es, opts.host_slices, opts.host_slices_w);
    }
    P->flops = 0;
    for (auto &st : P->steps) P->flops += st.flops;
    if (P->n_in == 2) P->flops_natural = P->flops;
    if (P->n_in == 1) P->flops_natural = 0;
    return COMET_OK;
}

void gemm_params_for(const std::vector<int64_t> &extent, const std::vector<int> &lm,
                     const std::vector<int> &ln, const std::vector<int> &lc, const Form &f,
                     GemmParams *g) {
    auto tm = label_strides(lm, extent), tn = label_strides(ln, extent), tc = label_strides(lc, extent);
    std::memset(g, 0, sizeof(*g));
    const int L = (int)extent.size();
    std::vector<int64_t> s0(L), s1(L);
    for (int l : f.M) { s0[l] = tm[l]; s1[l] = tc[l]; }
    fill_radix(&g->ma, f.M, extent.data(), s0.data(), s1.data());
    for (int l : f.N) { s0[l] = tn[l]; s1[l] = tc[l]; }
    fill_radix(&g->nb, f.N, extent.data(), s0.data(), s1.data());
    for (int l : f.K) { s0[l] = tm[l]; s1[l] = tn[l]; }
    fill_radix(&g->k, f.K, extent.data(), s0.data(), s1.data());
    g->M = (uint32_t)prod_ext(extent, f.M);
    g->N = (uint32_t)prod_ext(extent, f.N);
    g->K = (uint32_t)prod_ext(extent, f.K);
    g->ma.total = g->M; g->nb.total = g->N; g->k.total = g->K;
}

std::string describe_plan(const Plan &P) {
    std::ostringstream o;
    auto names = [&](const std::vector<int> &v) {
        std::string s = "[";
        for (size_t i = 0; i < v.size(); ++i) { if (i) s += ","; s += "\"" + P.label_names[v[i]] + "\""; }
        return s + "]";
    };
    o << "{\"expr\":\"" << P.expr << "\",\"dtype\":\"" << (P.dtype == COMET_F32 ? "f32" : "f64")
      << "\",\"precision\":\"" << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "split_bf16"
                                       : P.opts.precision == COMET_PREC_EMU_F64 ? "emu_f64" : "native")
      << "\",\"order\":\"" << P.tree << "\",\"flops\":" << P.flops << ",\"flops_natural\":" << P.flops_natural
      << ",\"workspace\":" << P.workspace << ",\"steps\":[";
    for (size_t i = 0; i < P.steps.size(); ++i) {
        const Step &s = P.steps[i];
        if (i) o << ",";
        o << "{\"kernel\":\"" << (s.kernel == KK_COPY ? "copy" : s.kernel == KK_GEMM_SPLIT ? "gemm_split_bf16"
                                    : s.kernel == KK_GEMM_EMU ? "gemm_emu_bf16x6"
                                    : s.kernel == KK_GEMV ? "gemv" : s.kernel == KK_REDUCE ? "reduce" : "gemm_f64")
          << "\",\"a\":" << s.a << ",\"b\":" << s.b << ",\"c\":" << s.c
          << ",\"a_labels\":" << names(P.slots[s.a].labels);
        if (s.b >= 0) o << ",\"b_labels\":" << names(P.slots[s.b].labels);
        o << ",\"c_labels\":" << names(P.slots[s.c].labels);
        if (s.kernel == KK_COPY)   // transpose engine: vector widths (negative out = copy mode), tile
            o << ",\"vec_in\":" << s.copy_vec_in << ",\"vec_out\":" << s.copy_vec_out << ",\"tile\":["
              << s.copy.tu << "," << s.copy.tv << "," << s.copy.tw << "]";
        if (s.kernel != KK_COPY) {
            o << ",\"swap\":" << s.form.swap << ",\"M\":" << names(s.form.M) << ",\"N\":" << names(s.form.N)
              << ",\"K\":" << names(s.form.K) << ",\"batch\":" << names(s.form.Bt)
              << ",\"n_forms\":" << s.n_forms << ",\"form_index\":" << s.form_index
              << ",\"cost_s\":" << s.form.cost << ",\"pre_bytes\":" << s.form.pre_bytes
              << ",\"eff_store\":" << s.form.eff_store << ",\"flops\":" << s.flops
              << ",\"ksplit\":" << s.ksplit;
            if (s.kernel == KK_GEMM_SPLIT)
                o << ",\"tail_tiles\":" << s.tail_tiles << ",\"tail_slices\":" << s.tail_slices;
        }
        o << "}";
    }
    o << "]";
    bool any_view = false;
    for (auto &sl : P.slots) any_view |= sl.view;
    if (any_view) {   // inputs (tensor = position) and the output (tensor = n_in) taken as views
        o << ",\"views\":[";
        bool first = true;
        for (auto &sl : P.slots) {
            if (!sl.view) continue;
            o << (first ? "" : ",") << "{\"tensor\":" << (sl.kind == SLOT_INPUT ? sl.index : P.n_in)
              << ",\"offset\":" << sl.offset << ",\"storage\":" << sl.storage << ",\"strides\":{";
            bool f2 = true;
            for (int l : sl.labels) {
                o << (f2 ? "" : ",") << "\"" << P.label_names[l] << "\":" << sl.strides.at(l);
                f2 = false;
            }
            o << "}}";
            first = false;
        }
        o << "]";
    }
    if (P.pipe.ok) {
        auto list = [&](const std::vector<int64_t> &v) {
            std::ostringstream l;
            l << "[";
            for (size_t k = 0; k < v.size(); ++k) l << (k ? "," : "") << v[k];
            l << "]";
            return l.str();
        };
        o << ",\"host_pipe\":{\"slices\":" << P.pipe.n_chunks << ",\"label\":\""
          << P.label_names[P.pipe.label] << "\",\"bounds\":" << list(P.pipe.xb) << ",\"side\":\""
          << (P.pipe.side ? "N" : "M") << "\",\"w_slices\":" << P.pipe.w_n << ",\"w_label\":\""
          << P.label_names[P.pipe.w_label] << "\",\"w_bounds\":" << list(P.pipe.wb)
          << ",\"blockwise\":" << (P.pipe.blockwise ? "true" : "false") << ",\"model_s\":[" << P.pipe.model_s[0] << ","
          << P.pipe.model_s[1] << "]}";
    }
    o << "}";
    return o.str();
}

}  // namespace comet

extern "C" comet_status_t comet_adjoint_expr(const char *expr, int operand, char *buf, size_t len) {
    if (!expr || !buf) return COMET_ERR_NULL;
    comet::ParsedExpr e;
    std::string err;
    comet_status_t st = comet::parse_expr(expr, &e, &err);
    if (st != COMET_OK) return st;
    if (e.op != 0) return COMET_ERR_UNSUPPORTED;
    if (operand < 0 || operand >= (int)e.ins.size()) return COMET_ERR_ARG;
    auto labels = [](const std::vector<std::string> &v) {
        std::string s = "[";
        for (size_t i = 0; i < v.size(); ++i) { if (i) s += ","; s += v[i]; }
        return s + "]";
    };
    std::ostringstream o;
    o.precision(17);
    o << "d" << e.ins[operand].name << labels(e.ins[operand].labels) << " = ";
    if (e.alpha != 1.0) o << e.alpha << " * ";
    o << "_G" << labels(e.out.labels);
    for (int t = 0; t < (int)e.ins.size(); ++t)
        if (t != operand) o << " * " << e.ins[t].name << labels(e.ins[t].labels);
    std::string s = o.str();
    if (s.size() + 1 > len) return COMET_ERR_ARG;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return COMET_OK;
}

extern "C" void comet_plan_opts_default(comet_plan_opts_t *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = COMET_PREC_NATIVE;
    o->order = COMET_ORDER_PLANNED;
    o->alpha = 1.0;
    o->workspace_cap = 0;
    o->form = -1;
    o->kc = 0;
    o->timeout_ms = 0;
    o->debug_flags = 0;
    o->ksplit = 0;
    o->host_slices = 0;
    o->host_slices_w = 0;
}
