// Host side of the batched plans: per-block descriptors, work-item prefix sums, the split
// path's plane layout, the workspace layout and the autotuner's cache.  No device code: the
// CPU replay of the batched kernels' index arithmetic (tests/batched_check.cpp) links it.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/comet.h"
#include "batched.h"

namespace comet {

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;
static bool g_tune_loaded = false;

static void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("COMET_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {   // one entry per line: "<cfg> <signature>"
        std::istringstream is(line);
        int c;
        std::string sig;
        if (is >> c && std::getline(is, sig) && !sig.empty()) g_tune_cache[sig.substr(1)] = c;
    }
}

static void tune_cache_store(const std::string &sig, int c) {
    g_tune_cache[sig] = c;
    const char *path = std::getenv("COMET_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << c << " " << sig << "\n";
}

// problem class: expression, dtype, precision, block count and the spread of block sizes
std::string batched_signature(const Plan &P) {
    std::ostringstream o;
    double fmin = 1e300, fmax = 0;
    for (size_t b = 0; b < P.block_flops.size(); ++b) {
        fmin = std::min(fmin, P.block_flops[b]);
        fmax = std::max(fmax, P.block_flops[b]);
    }
    o << P.expr << "|" << (P.dtype == COMET_F32 ? "f32" : "f64") << "|"
      << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "split" : "f64") << "|n=" << P.n_blocks
      << "|fmin=" << (long long)(fmin / 1e6) << "M|fmax=" << (long long)(fmax / 1e6) << "M";
    return o.str();
}

std::string describe_batched(const Plan &P) {
    std::ostringstream o;
    const TileCfg c = cfg_of(P, P.tile_cfg);
    o << "{\"batched\":true,\"expr\":\"" << P.expr << "\",\"n_blocks\":" << P.n_blocks
      << ",\"precision\":\"" << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "split_bf16" : "native")
      << "\",\"flops\":" << P.flops << ",\"workspace\":" << P.batched_ws << ",\"tile_cfg\":" << P.tile_cfg
      << ",\"tile\":[" << c.bm << "," << c.bn << "],\"n_tile_cfgs\":" << n_cfg(P)
      << ",\"a_kcontig\":" << P.batched_ak << ",\"b_kcontig\":" << P.batched_bk
      << ",\"swap\":" << P.batched_swap << ",\"dual_accumulators\":" << P.batched_dual
      << ",\"kernel\":\"" << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "tcgen05" : "mma_f64")
      << "\",\"plane_rows\":" << P.batched_plane_rows << ",\"signature\":\""
      << batched_signature(P) << "\"}";
    return o.str();
}

int tune_cache_lookup(const std::string &sig) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    auto it = g_tune_cache.find(sig);
    return it != g_tune_cache.end() ? it->second : -1;
}

void tune_cache_record(const std::string &sig, int c) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    tune_cache_store(sig, c);
}

comet_status_t build_batched_plan(const char *expr, int n_blocks, const char *const *label_names, int n_labels,
                                  const int64_t *extents, const comet_dtype_t *dtypes, int n_dtypes,
                                  const comet_plan_opts_t *opts, int tile_hint, Plan *out, std::string *err_out) {
    if (!expr || !label_names || !extents || !dtypes) return COMET_ERR_NULL;
    if (n_blocks < 1 || n_labels < 1 || n_labels > 16) return COMET_ERR_ARG;
    for (int l = 0; l < n_labels; ++l) if (!label_names[l]) return COMET_ERR_NULL;
    for (int64_t i = 0; i < (int64_t)n_blocks * n_labels; ++i) if (extents[i] <= 0) return COMET_ERR_SHAPE;
    Plan &P = *out;
    std::string &err = *err_out;
    std::vector<comet_extent_t> ex(n_labels);
    for (int l = 0; l < n_labels; ++l) ex[l] = comet_extent_t{label_names[l], extents[l]};
    comet_status_t st;
    try {
        st = build_plan(expr, ex.data(), n_labels, nullptr, 0, dtypes, n_dtypes, opts, &P, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
    }
    if (st == COMET_OK && (P.n_in != 2 || P.op != 0 || P.steps.size() != 1)) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take one two-operand \"=\" contraction";
    }
    if (st == COMET_OK && !P.steps[0].form.Bt.empty()) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take no batch labels (labels on both operands and the result)";
    }
    if (st == COMET_OK && (P.slots[0].view || P.slots[1].view || P.slots[2].view)) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take no repeated labels";
    }
    if (st == COMET_OK && P.opts.precision == COMET_PREC_EMU_F64) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take the native or the split precision";
    }
    if (st != COMET_OK) return st;
    // map the caller's label order to the plan's label ids
    std::vector<int> col(P.label_names.size(), -1);
    for (size_t id = 0; id < P.label_names.size(); ++id)
        for (int l = 0; l < n_labels; ++l)
            if (P.label_names[id] == label_names[l]) col[id] = l;
    for (int c : col)
        if (c < 0) { err = "a label of the expression has no extent column"; return COMET_ERR_LABEL; }
    const Step &s0 = P.steps[0];
    const Slot &sa = P.slots[s0.a], &sb = P.slots[s0.b], &sc = P.slots[s0.c];
    const Slot &sm = s0.form.swap ? sb : sa, &sn = s0.form.swap ? sa : sb;
    P.batched = true;
    P.n_blocks = n_blocks;
    P.block_flops.resize(n_blocks);
    std::vector<BlockDesc> desc(n_blocks);
    std::vector<int64_t> e(P.label_names.size());
    double flops = 0;
    for (int b = 0; b < n_blocks; ++b) {
        for (size_t id = 0; id < e.size(); ++id) e[id] = extents[(int64_t)b * n_labels + col[id]];
        GemmParams g;
        gemm_params_for(e, sm.labels, sn.labels, sc.labels, s0.form, &g);
        if ((uint64_t)g.M * g.N >= (1ull << 32) || g.K > 1024) {
            err = "a block's output exceeds 2^32 elements or its K exceeds 1024";
            return COMET_ERR_UNSUPPORTED;
        }
        BlockDesc &d = desc[b];
        std::memset(&d, 0, sizeof(d));
        d.ma = g.ma; d.nb = g.nb; d.k = g.k;
        d.M = g.M; d.N = g.N; d.K = g.K;
        d.index = (uint32_t)b;
        int64_t na = 1, nbv = 1;
        for (int l : sa.labels) na *= e[l];
        for (int l : sb.labels) nbv *= e[l];
        // the kernels read A = the M operand, B = the N operand; inputs are in expression order
        d.a_elems = s0.form.swap ? nbv : na;
        d.b_elems = s0.form.swap ? na : nbv;
        P.block_flops[b] = 2.0 * g.M * (double)g.N * g.K;
        flops += P.block_flops[b];
        if (b == 0) {
            P.batched_ak = g.k.n > 0 && g.k.s0[0] == 1;
            P.batched_bk = g.k.n > 0 && g.k.s1[0] == 1;
        }
    }
    P.batched_swap = s0.form.swap != 0;
    P.flops = flops;
    P.flops_natural = flops;
    // longest first
    std::vector<int> order(n_blocks);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P.block_flops[x] > P.block_flops[y]; });
    const int ncfg = n_cfg(P);
    // split path: each operand's planes as rows of 32 K values in one array, in launch order:
    // ceil(K/32) chunks x 3 planes x (rows rounded up to 256) rows per operand
    size_t parts = 0;
    int64_t prow = 0;
    P.batched_dual = false;
    if (P.opts.precision == COMET_PREC_SPLIT_BF16) {
        for (int i = 0; i < n_blocks; ++i) {
            BlockDesc &d = desc[order[i]];
            d.nk16 = (d.K + 15) / 16;
            d.m_pad = (d.M + 255) / 256 * 256;
            d.n_pad = (d.N + 255) / 256 * 256;
            const int64_t nkc = (d.K + 31) / 32;
            d.a_row0 = prow;
            prow += nkc * 3 * d.m_pad;
            d.b_row0 = prow;
            prow += nkc * 3 * d.n_pad;
            if (d.K > 32) P.batched_dual = true;
        }
        if (prow >= (int64_t(1) << 31)) {
            err = "the split planes exceed 2^31 rows of 32 values";
            return COMET_ERR_UNSUPPORTED;
        }
        parts = (size_t)prow * kBatchedPlaneRow;
    }
    P.batched_parts = parts;
    P.batched_plane_rows = prow;
    P.batched_prefix.assign(ncfg, std::vector<uint32_t>(n_blocks + 1, 0));
    for (int c = 0; c < ncfg; ++c) {
        const TileCfg tc = cfg_of(P, c);
        uint64_t acc = 0;
        for (int i = 0; i < n_blocks; ++i) {
            const BlockDesc &d = desc[order[i]];
            P.batched_prefix[c][i] = (uint32_t)acc;
            acc += (uint64_t)((d.N + tc.bn - 1) / tc.bn);   // one item per N strip
        }
        if (acc >= (1ull << 32)) {
            err = "more than 2^32 tiles";
            return COMET_ERR_UNSUPPORTED;
        }
        P.batched_prefix[c][n_blocks] = (uint32_t)acc;
    }
    // split path: one record per work item and configuration
    const bool split = P.opts.precision == COMET_PREC_SPLIT_BF16;
    P.batched_item_off.assign(ncfg, 0);
    size_t item_bytes = 0;
    for (int c = 0; c < ncfg && split; ++c) {
        P.batched_item_off[c] = item_bytes;
        item_bytes += ((size_t)P.batched_prefix[c][n_blocks] * sizeof(ItemRec) + 255) / 256 * 256;
    }
    P.batched_item_bytes = item_bytes;
    const BLayout L = layout_of(n_blocks, ncfg, item_bytes, parts);
    P.batched_ws = L.total;
    P.batched_table.assign(L.parts - L.prefix, 0);
    for (int c = 0; c < ncfg; ++c)
        std::memcpy(P.batched_table.data() + 4 * (size_t)c * (n_blocks + 1), P.batched_prefix[c].data(),
                    4 * (size_t)(n_blocks + 1));
    for (int i = 0; i < n_blocks; ++i)
        std::memcpy(P.batched_table.data() + (L.desc - L.prefix) + sizeof(BlockDesc) * (size_t)i, &desc[order[i]],
                    sizeof(BlockDesc));
    for (int c = 0; c < ncfg && split; ++c) {
        const TileCfg tc = cfg_of(P, c);
        ItemRec *rec = reinterpret_cast<ItemRec *>(P.batched_table.data() + (L.items - L.prefix) + P.batched_item_off[c]);
        for (int i = 0; i < n_blocks; ++i) {
            const BlockDesc &d = desc[order[i]];
            for (uint32_t it = P.batched_prefix[c][i]; it < P.batched_prefix[c][i + 1]; ++it) {
                ItemRec &r = rec[it];
                r.pos = (uint32_t)i;
                r.index = d.index;
                r.n0 = (it - P.batched_prefix[c][i]) * (uint32_t)tc.bn;
                r.mtiles = (d.M + tc.bm - 1) / tc.bm;
                r.nk16 = d.nk16;
                r.M = d.M;
                r.N = d.N;
                r.m_pad = d.m_pad;
                r.n_pad = d.n_pad;
                r.a_row0 = (int32_t)d.a_row0;
                r.b_row0 = (int32_t)d.b_row0;
                r.pad = 0;
            }
        }
    }
    if (tile_hint >= ncfg) return COMET_ERR_ARG;
    int cfg = tile_hint;
    if (cfg < 0) {
        const int c = tune_cache_lookup(batched_signature(P));
        cfg = (c >= 0 && c < ncfg) ? c : 0;
    }
    P.tile_cfg = cfg;
    return COMET_OK;
}

}  // namespace comet
