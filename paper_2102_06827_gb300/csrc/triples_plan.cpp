// Host side of the fused triples accumulation: the planner (terms, owned pair, block table,
// workspace) and the construction of the kernel's argument block.  No device code: the CPU
// replay of the kernel's index arithmetic (tests/triples_check.cpp) links it.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "triples.h"

namespace comet {

using namespace tri;


comet_status_t plan_triples(const char *const *terms, int n_terms, const char *const *names,
                                   int n_labels, int n_blocks, const int64_t *extents, const int *signs,
                                   comet_dtype_t dtype, Plan *P, std::string *err) {
    if (!terms || !names || !extents || !signs) return COMET_ERR_NULL;
    if (n_terms < 1 || n_terms > 16) { *err = "1 to 16 terms"; return COMET_ERR_ARG; }
    if (n_labels < 7 || n_labels > 16) { *err = "7 to 16 labels"; return COMET_ERR_ARG; }
    if (n_blocks < 1) { *err = "no blocks"; return COMET_ERR_ARG; }
    if (dtype != COMET_F32 && dtype != COMET_F64) { *err = "unknown dtype"; return COMET_ERR_DTYPE; }
    std::map<std::string, int> col;
    for (int l = 0; l < n_labels; ++l) {
        if (!names[l]) return COMET_ERR_NULL;
        if (col.count(names[l])) { *err = "label named twice"; return COMET_ERR_ARG; }
        col[names[l]] = l;
    }
    TriplesPlan &tp = P->tri;
    tp = TriplesPlan();
    tp.n_terms = n_terms;
    tp.n_labels = n_labels;
    tp.n_blocks = n_blocks;
    std::vector<std::string> tl;
    std::ostringstream all;
    for (int p = 0; p < n_terms; ++p) {
        if (!terms[p]) return COMET_ERR_NULL;
        ParsedExpr e;
        comet_status_t st = parse_expr(terms[p], &e, err);
        if (st != COMET_OK) return st;
        if (e.op != 0 || e.ins.size() != 2) { *err = "a term is T[...] = [alpha *] X[...] * Y[...]"; return COMET_ERR_UNSUPPORTED; }
        if (e.out.labels.size() != 6) { *err = "T has six labels"; return COMET_ERR_UNSUPPORTED; }
        if (p == 0) tl = e.out.labels;
        else if (e.out.labels != tl) { *err = "every term writes T with the same labels in the same order"; return COMET_ERR_LABEL; }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < i; ++j)
                if (tl[i] == tl[j]) { *err = "repeated label in T"; return COMET_ERR_UNSUPPORTED; }
        const auto &X = e.ins[0].labels, &Y = e.ins[1].labels;
        if (X.size() != 4 || Y.size() != 4) { *err = "operands have four labels"; return COMET_ERR_UNSUPPORTED; }
        TriTerm tt;
        tt.alpha = e.alpha;
        std::string dlab;
        int seen[6] = {0, 0, 0, 0, 0, 0};
        for (int side = 0; side < 2; ++side) {
            const auto &L = side ? Y : X;
            const auto &O = side ? X : Y;
            for (int m = 0; m < 4; ++m) {
                if (!col.count(L[m])) { *err = "label " + L[m] + " has no extent column"; return COMET_ERR_LABEL; }
                int q = -1;
                for (int i = 0; i < 6; ++i) if (tl[i] == L[m]) q = i;
                const bool on_other = std::find(O.begin(), O.end(), L[m]) != O.end();
                if (q < 0) {
                    if (!on_other) { *err = "label " + L[m] + " is on one operand only and not on T"; return COMET_ERR_UNSUPPORTED; }
                    if (!dlab.empty() && dlab != L[m]) { *err = "a term sums exactly one label"; return COMET_ERR_UNSUPPORTED; }
                    dlab = L[m];
                } else {
                    if (on_other) { *err = "a label of T on both operands"; return COMET_ERR_UNSUPPORTED; }
                    ++seen[q];
                }
                (side ? tt.y_q : tt.x_q)[m] = q;
                (side ? tt.y_col : tt.x_col)[m] = col[L[m]];
            }
        }
        if (dlab.empty()) { *err = "a term sums exactly one label"; return COMET_ERR_UNSUPPORTED; }
        int cx = 0;
        for (int m = 0; m < 4; ++m) cx += tt.x_q[m] < 0;
        if (cx != 1) { *err = "the summed label appears once per operand"; return COMET_ERR_UNSUPPORTED; }
        for (int q = 0; q < 6; ++q)
            if (seen[q] != 1) { *err = "every label of T on exactly one operand"; return COMET_ERR_UNSUPPORTED; }
        tt.d_col = col[dlab];
        tp.terms.push_back(tt);
        all << (p ? " ; " : "") << terms[p];
    }
    for (int q = 0; q < 6; ++q) {
        if (!col.count(tl[q])) { *err = "label " + tl[q] + " has no extent column"; return COMET_ERR_LABEL; }
        tp.t_col[q] = col[tl[q]];
        if (signs[q] != 1 && signs[q] != -1) { *err = "signs are +1 or -1"; return COMET_ERR_ARG; }
        tp.signs[q] = signs[q];
    }
    // owned pair: the two T labels that sit on different operands in the most terms
    int best = -1;
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            int split = 0;
            for (auto &tt : tp.terms) {
                bool ix = false, jx = false;
                for (int m = 0; m < 4; ++m) { ix |= tt.x_q[m] == i; jx |= tt.x_q[m] == j; }
                split += ix != jx;
            }
            if (split > best) { best = split; tp.own[0] = i; tp.own[1] = j; }
        }
    // block table
    tp.ext.resize((size_t)n_blocks * n_labels);
    tp.prefix.assign(n_blocks + 1, 0);
    double flops = 0;
    for (int b = 0; b < n_blocks; ++b) {
        int64_t tiles = 1;
        double tel = 1;
        for (int l = 0; l < n_labels; ++l) {
            const int64_t x = extents[(size_t)b * n_labels + l];
            if (x < 1 || x > (1 << 30)) { *err = "extents between 1 and 2^30"; return COMET_ERR_SHAPE; }
            tp.ext[(size_t)b * n_labels + l] = (int32_t)x;
        }
        for (int q = 0; q < 6; ++q) {
            const int64_t x = extents[(size_t)b * n_labels + tp.t_col[q]];
            tiles *= (x + TS - 1) / TS;
            tel *= (double)x;
            if (tiles >= (1ll << 31)) { *err = "a block of 2^31 tiles or more"; return COMET_ERR_SHAPE; }
        }
        for (auto &tt : tp.terms) {
            flops += 2.0 * tel * (double)extents[(size_t)b * n_labels + tt.d_col];
            for (int side = 0; side < 2; ++side) {   // 32-bit element offsets inside every operand
                long double n = 1;
                for (int m = 0; m < 4; ++m) n *= (long double)extents[(size_t)b * n_labels + (side ? tt.y_col : tt.x_col)[m]];
                if (n >= 2147483648.0L) { *err = "an operand of 2^31 elements or more"; return COMET_ERR_SHAPE; }
            }
        }
        tp.prefix[b + 1] = tp.prefix[b] + tiles;
    }
    size_t off = 0;
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    tp.ws_ext = off;
    off = align(off + tp.ext.size() * sizeof(int32_t));
    tp.ws_prefix = off;
    off = align(off + tp.prefix.size() * sizeof(int64_t));
    tp.ws_counter = off;
    off = align(off + 8);
    P->triples = true;
    P->batched = false;
    if (dtype == COMET_F32) plan_triples_tc(P);
    if (!tp.tc_batch.empty()) {
        off = align(off);
        tp.ws_tc_prefix = off;
        off = align(off + tp.tc_prefix.size() * sizeof(int64_t));
        tp.ws_tc_row0 = off;
        off = align(off + tp.tc_row0.size() * sizeof(int32_t));
        tp.ws_tc_rec = off;
        off = align(off + tp.tc_rec.size() * sizeof(int32_t));
        tp.ws_tc_planes = off;
        off = align(off + (size_t)tp.tc_max_rows * tc::ROWB);
    }
    P->workspace = off;
    P->dtype = dtype;
    P->flops = flops;
    P->flops_natural = flops;
    P->expr = all.str();
    return COMET_OK;
}

int64_t tc_operand_rows(const int *q, const int64_t *ext_t, int64_t ext_d) {
    int64_t tiles = 1;
    bool wide = false;
    for (int m = 0; m < 4; ++m) {
        if (q[m] < 0) continue;
        const int64_t ts = q[m] == 0 ? tc::WA : TS;
        tiles *= (ext_t[q[m]] + ts - 1) / ts;
        wide |= q[m] == 0;
    }
    const int64_t chunks = (ext_d + tc::KCH - 1) / tc::KCH;
    return tiles * chunks * 3 * (wide ? tc::WROWS : tc::NROWS);
}

void plan_triples_tc(Plan *P) {
    TriplesPlan &tp = P->tri;
    // plane rows per batch: MAX_BATCH_ROWS, or less from COMET_TRIPLES_BATCH_ROWS (more batches;
    // a block larger than a batch puts the plan on the FMA kernel)
    int64_t cap = tc::MAX_BATCH_ROWS;
    if (const char *env = std::getenv("COMET_TRIPLES_BATCH_ROWS")) {
        const long long v = std::atoll(env);
        if (v > 0 && v < cap) cap = v;
    }
    const int nb = tp.n_blocks, nt = tp.n_terms, nl = tp.n_labels;
    tp.tc_prefix.assign(nb + 1, 0);
    tp.tc_row0.assign((size_t)nb * nt * 2, 0);
    tp.tc_rows.assign(nb, 0);
    tp.tc_rec.clear();
    tp.tc_rec.reserve((size_t)nb * nt * 16);
    tp.tc_batch.clear();
    tp.tc_max_rows = 0;
    int64_t batch_rows = 0;
    for (int b = 0; b < nb; ++b) {
        int64_t ext_t[6];
        for (int q = 0; q < 6; ++q) ext_t[q] = tp.ext[(size_t)b * nl + tp.t_col[q]];
        int64_t items = (ext_t[0] + tc::WA - 1) / tc::WA;
        for (int q = 1; q < 6; ++q) items *= (ext_t[q] + TS - 1) / TS;
        tp.tc_prefix[b + 1] = tp.tc_prefix[b] + items;
        int64_t rows = 0;
        for (int p = 0; p < nt; ++p) {
            const TriTerm &tt = tp.terms[p];
            const int64_t ed = tp.ext[(size_t)b * nl + tt.d_col];
            rows += tc_operand_rows(tt.x_q, ext_t, ed) + tc_operand_rows(tt.y_q, ext_t, ed);
        }
        tp.tc_rows[b] = rows;
        if (rows > cap) {   // a block too large for one batch: the FMA kernel runs the plan
            tp.tc_batch.clear();
            tp.tc_max_rows = 0;
            return;
        }
        if (tp.tc_batch.empty() || batch_rows + rows > cap) {
            tp.tc_batch.push_back(b);
            batch_rows = 0;
        }
        for (int p = 0; p < nt; ++p) {   // operands of the block in order, from its batch's start
            const TriTerm &tt = tp.terms[p];
            const int64_t ed = tp.ext[(size_t)b * nl + tt.d_col];
            tp.tc_row0[((size_t)b * nt + p) * 2] = (int32_t)batch_rows;
            batch_rows += tc_operand_rows(tt.x_q, ext_t, ed);
            tp.tc_row0[((size_t)b * nt + p) * 2 + 1] = (int32_t)batch_rows;
            batch_rows += tc_operand_rows(tt.y_q, ext_t, ed);
        }
        tp.tc_max_rows = std::max(tp.tc_max_rows, batch_rows);
        // the block's term records: plane row of each operand tile as a linear form in the
        // pair-tile coordinates
        for (int p = 0; p < nt; ++p) {
            const TriTerm &tt = tp.terms[p];
            const int64_t ed = tp.ext[(size_t)b * nl + tt.d_col];
            const int64_t nch = (ed + tc::KCH - 1) / tc::KCH;
            TcRec r;
            std::memset(&r, 0, sizeof(r));
            r.nch = (int32_t)nch;
            r.ed = (int32_t)ed;
            bool x_wide = false;
            for (int m = 0; m < 4; ++m) x_wide |= tt.x_q[m] == 0;
            for (int w = 0; w < 2; ++w) {
                const int side = (w == 0) == x_wide ? 0 : 1;
                const int *q = side ? tt.y_q : tt.x_q;
                r.row0[w] = tp.tc_row0[((size_t)b * nt + p) * 2 + side];
                int lab[3], k = 0;
                for (int l = 0; l < 6; ++l)
                    for (int m = 0; m < 4; ++m)
                        if (q[m] == l) lab[k++] = l;
                int64_t step = nch * 3 * (w == 0 ? tc::WROWS : tc::NROWS);
                for (int i = 0; i < 3; ++i) {
                    r.coef[w][lab[i]] = (int32_t)step;
                    const int64_t ts = lab[i] == 0 ? tc::WA : TS;
                    step *= (ext_t[lab[i]] + ts - 1) / ts;
                }
            }
            const int32_t *rw = reinterpret_cast<const int32_t *>(&r);
            tp.tc_rec.insert(tp.tc_rec.end(), rw, rw + 16);
        }
    }
    tp.tc_batch.push_back(nb);
}

std::string describe_triples(const Plan &P) {
    const TriplesPlan &tp = P.tri;
    std::ostringstream o;
    o.precision(17);
    o << "{\"triples\":true,\"terms\":" << tp.n_terms << ",\"blocks\":" << tp.n_blocks
      << ",\"dtype\":\"" << (P.dtype == COMET_F32 ? "f32" : "f64") << "\",\"tiles\":" << tp.prefix.back()
      << ",\"tile\":[4,4,4,4,4,4],\"own\":[" << tp.own[0] << "," << tp.own[1] << "],\"flops\":" << P.flops
      << ",\"workspace\":" << P.workspace << ",\"tensor_core\":" << (tp.tc_batch.empty() ? "false" : "true");
    if (!tp.tc_batch.empty())
        o << ",\"pair_tiles\":" << tp.tc_prefix.back() << ",\"batches\":" << tp.tc_batch.size() - 1
          << ",\"plane_rows\":" << tp.tc_max_rows;
    o << "}";
    return o.str();
}

void triples_args(const Plan &P, Args *out) {
    const TriplesPlan &tp = P.tri;
    Args &a = *out;
    std::memset(&a, 0, sizeof(a));
    a.n_terms = tp.n_terms;
    a.n_labels = tp.n_labels;
    a.n_blocks = tp.n_blocks;
    int nf = 0;
    for (int q = 0; q < 6; ++q) {
        a.t_col[q] = (int8_t)tp.t_col[q];
        if (q != tp.own[0] && q != tp.own[1]) {
            a.fixed_sign[nf] = (float)tp.signs[q];
            a.fixed[nf++] = (int8_t)q;
        }
    }
    for (int j = 0; j < 2; ++j) {
        a.own[j] = (int8_t)tp.own[j];
        a.own_sign[j] = (float)tp.signs[tp.own[j]];
    }
    for (int q = 0; q < 6; ++q) a.sign[q] = (float)tp.signs[q];
    for (int p = 0; p < tp.n_terms; ++p) {
        const TriTerm &tt = tp.terms[p];
        a.term[p].alpha = tt.alpha;
        a.term[p].amode = (int8_t)(tt.alpha == 1.0 ? 0 : tt.alpha == -1.0 ? 1 : 2);
        for (int m = 0; m < 4; ++m) {
            a.term[p].x_q[m] = (int8_t)tt.x_q[m];
            a.term[p].y_q[m] = (int8_t)tt.y_q[m];
            a.term[p].x_col[m] = (int8_t)tt.x_col[m];
            a.term[p].y_col[m] = (int8_t)tt.y_col[m];
        }
        a.term[p].d_col = (int8_t)tt.d_col;
        int xmask = 0;
        for (int m = 0; m < 4; ++m) if (tt.x_q[m] >= 0) xmask |= 1 << tt.x_q[m];
        a.term[p].xmask = (int8_t)xmask;
        for (int side = 0; side < 2; ++side) {   // rank of each dimension's T label in T order
            const int *q = side ? tt.y_q : tt.x_q;
            int8_t *rk = side ? a.term[p].y_rank : a.term[p].x_rank;
            for (int m = 0; m < 4; ++m) {
                rk[m] = -1;
                if (q[m] < 0) continue;
                int r = 0;
                for (int n = 0; n < 4; ++n) r += q[n] >= 0 && q[n] < q[m];
                rk[m] = (int8_t)r;
            }
        }
        // tile digits: the owned labels an operand holds come first (own[0], then own[1]), so
        // that they run along consecutive shared-memory entries; then its fixed labels
        for (int side = 0; side < 2; ++side) {
            const int *q = side ? tt.y_q : tt.x_q;
            int8_t *dig = side ? a.term[p].y_dig : a.term[p].x_dig;
            int nd = 0;
            for (int m = 0; m < 4; ++m) dig[m] = -1;
            for (int o = 0; o < 2; ++o)
                for (int m = 0; m < 4; ++m) if (q[m] == tp.own[o]) dig[m] = (int8_t)nd++;
            for (int m = 0; m < 4; ++m) if (q[m] >= 0 && dig[m] < 0) dig[m] = (int8_t)nd++;
        }
    }
}

}  // namespace comet
