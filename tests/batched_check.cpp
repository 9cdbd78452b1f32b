// CPU replay of the index arithmetic of the tensor-core batched kernel (k_batched_tc.cu) and
// its split pre-pass, on the descriptor tables the real planner builds (batched_plan.cpp).
// Checks, for many random block tables (uneven extents, K from 1 to 1024, degenerate blocks)
// and both strip widths:
//   - the pre-pass writes every plane row of the plane region exactly once, inside its buffer;
//   - every TMA box the producer loads lies inside the chunk-plane of the operand it names,
//     inside the plane region, with int32 coordinates; every shared-memory destination lies
//     inside its strip slot or ring slot on a 1024-byte boundary;
//   - the rows an MMA tile reads beyond M (columns beyond N) are padding rows the pre-pass
//     zeroed, so out-of-range outputs are exactly zero;
//   - tensor-memory columns stay below the 512 allocated; shared memory fits the opt-in limit;
//   - the epilogue's output offsets (row part + column part) hit every element of a block's
//     output exactly once, and the weight's row/column parts split the output offset into the
//     first operand's labels and the second operand's labels.
// Built and run by tests/test_index_check.py; exit status 0 = pass.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../paper_2102_06827_gb300/csrc/batched.h"

using namespace comet;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

// the kernel's work-item lookup (prefix[pos] <= it < prefix[pos + 1])
static uint32_t find_block(const uint32_t *prefix, uint32_t n_blocks, uint32_t it) {
    uint32_t lo = 0, hi = n_blocks;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= it) lo = mid; else hi = mid;
    }
    return lo;
}

static void check_plan(const char *expr, const std::vector<std::vector<int64_t>> &ext) {
    const char *names[7] = {"a", "b", "c", "i", "j", "k", "d"};
    const int nb = (int)ext.size();
    std::vector<int64_t> flat;
    for (auto &r : ext) flat.insert(flat.end(), r.begin(), r.end());
    comet_plan_opts_t o;
    comet_plan_opts_default(&o);
    o.precision = COMET_PREC_SPLIT_BF16;
    comet_dtype_t dt[3] = {COMET_F32, COMET_F32, COMET_F32};
    Plan P;
    std::string err;
    comet_status_t st = build_batched_plan(expr, nb, names, 7, flat.data(), dt, 3, &o, 0, &P, &err);
    CHECK(st == COMET_OK, "plan failed: %s", err.c_str());
    if (st != COMET_OK) return;
    const BLayout L = layout_of(nb, n_cfg(P), P.batched_item_bytes, P.batched_parts);
    CHECK(L.parts % 256 == 0, "plane region alignment");
    CHECK(P.batched_parts == (size_t)P.batched_plane_rows * kBatchedPlaneRow, "plane bytes");
    CHECK(P.batched_plane_rows < (int64_t(1) << 31), "plane rows above int32");
    const BlockDesc *desc = reinterpret_cast<const BlockDesc *>(P.batched_table.data() + (L.desc - L.prefix));
    bool any_dual = false;
    // ---- pre-pass: every plane row written once ----
    std::vector<uint8_t> written((size_t)P.batched_plane_rows, 0);
    for (int i = 0; i < nb; ++i) {
        const BlockDesc &d = desc[i];
        CHECK(d.nk16 == (d.K + 15) / 16 && d.nk16 * 16 <= 1024, "nk16");
        CHECK(d.m_pad % 256 == 0 && d.m_pad >= d.M && d.n_pad % 256 == 0 && d.n_pad >= d.N, "padding");
        if (d.K > 32) any_dual = true;
        const uint32_t nkc = (d.K + 31) / 32;   // chunks of 32 K values, one plane row each
        CHECK(nkc * 32 <= 1024, "pre-pass offset table");
        for (int op = 0; op < 2; ++op) {
            const int64_t r0 = op ? d.b_row0 : d.a_row0;
            const uint32_t pad = op ? d.n_pad : d.m_pad;
            const int64_t n = (int64_t)nkc * 3 * pad;
            CHECK(r0 >= 0 && r0 + n <= P.batched_plane_rows, "operand planes outside the region");
            for (int64_t r = r0; r < r0 + n && r < P.batched_plane_rows; ++r) {
                CHECK(!written[r], "plane row %lld written twice", (long long)r);
                written[r] = 1;
            }
        }
    }
    for (int64_t r = 0; r < P.batched_plane_rows; ++r) CHECK(written[r], "plane row %lld never written", (long long)r);
    CHECK(any_dual == P.batched_dual, "dual flag");
    // ---- tensor memory and shared memory ----
    CHECK(btc::Cfg<256>::SMEM <= 232448 && btc::Cfg<128>::SMEM <= 232448, "shared memory above 227 KB");
    for (int c = 0; c < n_cfg(P); ++c) {
        const int BN = cfg_of(P, c).bn;
        CHECK(BN == 128 || BN == 256, "strip width");
        const uint32_t buf_cols = P.batched_dual ? 2 * BN : BN, nbuf = btc::TMEM_COLS / buf_cols;
        CHECK(nbuf >= 1 && nbuf <= 4, "tensor-memory buffers");
        // highest column the MMA writes / the epilogue reads: last buffer + P1 + last column
        const uint32_t top = (nbuf - 1) * buf_cols + (P.batched_dual ? BN : 0) + BN;
        CHECK(top <= btc::TMEM_COLS, "tensor-memory columns %u", top);
        const int strip_bytes = 3 * BN * btc::ROW;
        const uint32_t *prefix = P.batched_prefix[c].data();
        const uint32_t n_items = prefix[nb];
        const int halves = BN / btc::BOX_ROWS;
        CHECK(P.batched_item_off[c] + (size_t)n_items * sizeof(ItemRec) <= P.batched_item_bytes, "item records");
        const ItemRec *items = reinterpret_cast<const ItemRec *>(P.batched_table.data() + (L.items - L.prefix) +
                                                                 P.batched_item_off[c]);
        CHECK(((L.items + P.batched_item_off[c]) % 16) == 0, "item records not 16-byte aligned");
        for (uint32_t it = 0; it < n_items; ++it) {
            const uint32_t pos = find_block(prefix, (uint32_t)nb, it);
            CHECK(prefix[pos] <= it && it < prefix[pos + 1], "item lookup");
            const BlockDesc &d = desc[pos];
            const ItemRec &rec = items[it];
            // the record the kernel reads agrees with the prefix sums and the descriptor
            CHECK(rec.pos == pos && rec.index == d.index && rec.n0 == (it - prefix[pos]) * BN &&
                  rec.mtiles == (d.M + btc::BM - 1) / btc::BM && rec.nk16 == d.nk16 && rec.M == d.M &&
                  rec.N == d.N && rec.m_pad == d.m_pad && rec.n_pad == d.n_pad && rec.a_row0 == d.a_row0 &&
                  rec.b_row0 == d.b_row0, "item record %u", it);
            const uint32_t n0 = rec.n0;
            CHECK(n0 < d.N, "strip beyond N");
            const uint32_t mtiles = rec.mtiles;
            const bool res = d.nk16 <= (uint32_t)btc::MAX_RES_NK;
            CHECK(res || P.batched_dual, "streamed B without dual accumulators");
            auto box = [&](int64_t row0, uint32_t pad, uint32_t kc, uint32_t r0, uint32_t limit) {
                const int64_t lo = row0 + (int64_t)(kc * 3) * pad, y = lo + r0;   // plane 0; planes 1, 2 follow
                for (uint32_t p = 0; p < 3; ++p) {
                    const int64_t yp = y + (int64_t)p * pad, lop = lo + (int64_t)p * pad;
                    CHECK(yp >= lop && yp + btc::BOX_ROWS <= lop + pad, "box outside its chunk-plane");
                    CHECK(yp + btc::BOX_ROWS <= P.batched_plane_rows && yp <= INT32_MAX, "box outside the region");
                }
                CHECK(r0 + btc::BOX_ROWS <= pad, "box rows beyond the padded rows");
                CHECK(r0 < limit, "box starts beyond the operand's rows");
            };
            const uint32_t nkc = (d.nk16 + 1) / 2;
            CHECK(!res || nkc == 1, "a resident strip holds one chunk");
            if (res) {
                for (uint32_t p = 0; p < 3; ++p)
                    for (int h = 0; h < halves; ++h) {
                        const int off = (int)(p * BN + h * btc::BOX_ROWS) * btc::ROW;
                        CHECK(off % 1024 == 0 && off + btc::BOX_BYTES <= strip_bytes, "strip destination");
                    }
                // (the second half of a 256-wide strip may lie wholly in the zero padding)
                for (int h = 0; h < halves; ++h) box(d.b_row0, d.n_pad, 0, n0 + h * btc::BOX_ROWS, d.n_pad);
            }
            // a ring slot holds three 128-row plane boxes; the MMA's second K step reads 32 bytes
            // into each 64-byte row
            CHECK(btc::SLOT_BYTES == 3 * btc::BOX_BYTES && btc::BOX_BYTES % 1024 == 0 && 32 + 32 <= btc::ROW,
                  "slot geometry");
            for (uint32_t mt = 0; mt < mtiles; ++mt)
                for (uint32_t kc = 0; kc < nkc; ++kc) {
                    box(d.a_row0, d.m_pad, kc, mt * btc::BM, d.M);
                    if (!res)
                        for (int h = 0; h < halves; ++h) box(d.b_row0, d.n_pad, kc, n0 + h * btc::BOX_ROWS, d.n_pad);
                }
        }
    }
    // ---- epilogue offsets: every output element once; weight parts by operand ----
    const Step &s0 = P.steps[0];
    const Slot &sc = P.slots[s0.c];
    for (int i = 0; i < nb; ++i) {
        const BlockDesc &d = desc[i];
        const uint64_t n_out = (uint64_t)d.M * d.N;
        if (n_out > (1u << 22)) continue;   // the small blocks give full coverage quickly
        std::vector<uint8_t> hit(n_out, 0);
        std::vector<int64_t> orow(d.M), ocol(d.N);
        for (uint32_t m = 0; m < d.M; ++m) { int64_t a, b; radix_offsets(d.ma, m, a, b); orow[m] = b; }
        for (uint32_t n = 0; n < d.N; ++n) { int64_t a, b; radix_offsets(d.nb, n, a, b); ocol[n] = b; }
        for (uint32_t m = 0; m < d.M; ++m)
            for (uint32_t n = 0; n < d.N; ++n) {
                const int64_t o = orow[m] + ocol[n];
                CHECK(o >= 0 && (uint64_t)o < n_out, "output offset out of range");
                if (o >= 0 && (uint64_t)o < n_out) { CHECK(!hit[o], "output written twice"); hit[o] = 1; }
            }
        // the row part of the offset uses only the M operand's labels: decompose it back
        const std::vector<int> &out_labels = sc.labels;
        const Slot &sm = s0.form.swap ? P.slots[s0.b] : P.slots[s0.a];
        const int64_t *ex = &flat[(size_t)d.index * 7];
        for (uint32_t m = 0; m < d.M; m += 7) {
            int64_t r = orow[m];
            for (int l : out_labels) {
                const int64_t e = ex[std::find(names, names + 7, P.label_names[l]) - names];
                const int64_t digit = r % e;
                r /= e;
                const bool in_m = std::find(sm.labels.begin(), sm.labels.end(), l) != sm.labels.end();
                CHECK(in_m || digit == 0, "row offset carries a label of the other operand");
            }
        }
    }
}

int main() {
    std::mt19937_64 rng(20260);
    const char *exprs[] = {"T[a,b,c,i,j,k] = A[d,a,b,i] * B[c,d,j,k]", "T[c,j,k,a,b,i] = A[d,a,b,i] * B[c,d,j,k]",
                           "T[a,c,i,j,b,k] = A[a,b,i,d] * B[d,c,j,k]"};
    int cases = 0;
    for (const char *e : exprs) {
        for (int rep = 0; rep < 6; ++rep) {
            std::vector<std::vector<int64_t>> ext;
            const int n = 1 + (int)(rng() % 40);
            for (int b = 0; b < n; ++b) {
                std::vector<int64_t> r(7);
                for (int l = 0; l < 6; ++l) r[l] = 1 + (int64_t)(rng() % (rep < 3 ? 33 : 12));
                const int kind = (int)(rng() % 6);
                r[6] = kind == 0 ? 1 + (int64_t)(rng() % 1024) : kind == 1 ? 33 + (int64_t)(rng() % 64)
                                                                    : 1 + (int64_t)(rng() % 32);
                if (rep == 5) r = {1, 1, 1, 1, 1, 1, 1 + (int64_t)(rng() % 40)};
                ext.push_back(r);
            }
            check_plan(e, ext);
            ++cases;
        }
        // the workload's shape class: extents 8..32, K <= 32 (one accumulator, resident strips)
        std::vector<std::vector<int64_t>> w;
        for (int b = 0; b < 64; ++b) {
            std::vector<int64_t> r(7);
            for (int l = 0; l < 7; ++l) r[l] = 8 + (int64_t)(rng() % 25);
            w.push_back(r);
        }
        check_plan(e, w);
        ++cases;
    }
    std::printf("%d plans, %d failures\n", cases, fails);
    return fails ? 1 : 0;
}
