// CPU replay of the index arithmetic of the fused triples kernels (k_triples.cu) on the argument
// block the real host code builds (triples_plan.cpp): the FP64 kernel (256 threads, thread tiles
// of 4 x 4, 16 summed values per step) and the FP32 kernel (64 threads, 2^6 elements per
// thread, 32 summed values per step).  Terms, labels, signs and one block's extents come from
// the command line: argv = n_terms, the terms, the 7 label names, 6 signs, 7 extents.
// FP32 kernel, for every term, thread and a set of tiles that includes the first and the ragged
// last tile along every label:
//   - thread r stages row r of each operand tile (rows inside the block only) from the operand
//     elements at the row's coordinates (global reads inside the operand): the operand holding
//     T label 0 into P [16][64], the other one into B [16][64];
//   - for every element inside the block, the X and Y entries the products read (row 8 h + x of
//     the thread's group) are the ones staged from the operands at that element's coordinates,
//     and the 64 (x, y) pairs of a summed index cover the thread's 64 elements once each; the
//     packed accumulator pairs (e, e + 1) take entries 2m and 2m + 1 of the operand holding T
//     label 0;
//   - the 16-byte shared loads start on 16-byte boundaries and stay in the tile.
// FP32 tensor-core path: the pair-tile layout in shared memory (one slot per element, the
// drained rows of a warp in 32 banks), batches and operand plane-row segments, the TMA boxes of
// every term and chunk inside their operand's segment, the drain's (row, column) -> element map
// against the elements' coordinates (each of the 8192 once), the pre-pass's plane rows against
// the operand elements, and the energy's element coverage.
// FP64 kernel:
// For every thread, every term and a set of tiles that includes the first and the ragged last
// tile along every label, it checks:
//   - the staging entries (kk, r) of stage_async stay inside the [kc][RP] shared tile, and the
//     global element offsets they read lie inside the operand (all digits guarded by rem);
//   - the 16-byte shared loads of step_compute start on 16-byte boundaries and stay in the row;
//   - the energy epilogue's eps reads stay inside the eps vectors;
//   - the static shared arrays the 16-byte loads use have 16-byte-multiple row pitches.
// Exit status 0 = pass.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_2102_06827_gb300/csrc/triples.h"

using namespace comet;
using namespace comet::tri;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

// the kernel's entry(): staging entry idx -> (kk, r)
static void entry(int KCt, int idx, int &kk, int &r) {
    const int hb = KCt / 8 == 4 ? 2 : 1;
    const int rest = idx >> 5;
    kk = ((rest & (KCt / 8 - 1)) << 3) | (idx & 7);
    r = ((rest >> hb) << 2) | ((idx >> 3) & 3);
}

struct TA { int base, sd, s[3], rem[3]; };

// the kernel's tile_addr(), with the element count of the operand it addresses
static TA tile_addr(const int8_t *q, const int8_t *col, const int8_t *dig, const int32_t *ext_b, const int *tbase,
                    const int *text, int k0, int64_t *n_elems) {
    TA ta{};
    int st = 1;
    for (int m = 0; m < 4; ++m) {
        if (q[m] < 0) {
            ta.sd = st;
            ta.base += k0 * st;
        } else {
            const int b0 = tbase[q[m]];
            const int rm = std::min(TS, text[q[m]] - b0);
            ta.base += b0 * st;
            if (dig[m] == 0) { ta.s[0] = st; ta.rem[0] = rm; }
            if (dig[m] == 1) { ta.s[1] = st; ta.rem[1] = rm; }
            if (dig[m] == 2) { ta.s[2] = st; ta.rem[2] = rm; }
        }
        st *= ext_b[col[m]];
    }
    *n_elems = st;
    return ta;
}

static void replay(const Args &a, const int32_t *ext_b, int elem) {
    const int kc = elem == 4 ? KC : KC / 2, RS = NT / kc, NIT = kc * R / NT;
    CHECK(RS == 8 || RS == 16, "lane pattern");
    CHECK((RP * elem) % 16 == 0, "row pitch of the staged tiles not a multiple of 16 bytes");
    int text[6], ntile[6];
    for (int q = 0; q < 6; ++q) {
        text[q] = ext_b[a.t_col[q]];
        ntile[q] = (text[q] + TS - 1) / TS;
    }
    // tiles: every combination of the first and the last tile along each label
    for (int mask = 0; mask < 64; ++mask) {
        int tbase[6];
        for (int q = 0; q < 6; ++q) tbase[q] = ((mask >> q) & 1) ? (ntile[q] - 1) * TS : 0;
        for (int t = 0; t < NT; ++t) {
            int f[4];
            for (int j = 0; j < 4; ++j) f[j] = (t >> (2 * j)) & 3;
            bool fixed_ok = true;
            for (int j = 0; j < 4; ++j) fixed_ok &= tbase[a.fixed[j]] + f[j] < text[a.fixed[j]];
            for (int p = 0; p < a.n_terms; ++p) {
                const TermDev &tm = a.term[p];
                const int K = ext_b[tm.d_col];
                // s_dig: rx, ry and the case, as the kernel forms them
                int rx = 0, ry = 0;
                bool u_on_x = false, v_on_x = false;
                for (int m = 0; m < 4; ++m) {
                    for (int j = 0; j < 4; ++j) {
                        if (tm.x_q[m] == a.fixed[j]) rx += f[j] << (2 * tm.x_dig[m]);
                        if (tm.y_q[m] == a.fixed[j]) ry += f[j] << (2 * tm.y_dig[m]);
                    }
                    u_on_x |= tm.x_q[m] == a.own[0];
                    v_on_x |= tm.x_q[m] == a.own[1];
                }
                const int kase = u_on_x ? (v_on_x ? 2 : 0) : (v_on_x ? 1 : 3);
                CHECK(rx < 64 && ry < 64, "row offsets above 6 bits");
                // 16-byte shared loads of step_compute: (row start, elements read)
                auto vec_load = [&](int r) {
                    CHECK((r * elem) % 16 == 0, "misaligned 16-byte shared load (term %d, r %d)", p, r);
                    CHECK(r + 4 <= R, "shared load beyond the row");
                };
                if (kase == 0) { vec_load(rx); vec_load(ry); }
                else if (kase == 1) { vec_load(ry); vec_load(rx); }
                else if (kase == 2) { for (int v = 0; v < 4; ++v) vec_load(rx + 4 * v); CHECK(ry < R, "scalar load"); }
                else { for (int v = 0; v < 4; ++v) vec_load(ry + 4 * v); CHECK(rx < R, "scalar load"); }
                (void)fixed_ok;
                // staging of every step of this term
                for (int k0 = 0; k0 < K; k0 += kc) {
                    const int kn = std::min(kc, K - k0);
                    for (int side = 0; side < 2; ++side) {
                        int64_t n_el = 0;
                        const TA ta = side ? tile_addr(tm.y_q, tm.y_col, tm.y_dig, ext_b, tbase, text, k0, &n_el)
                                           : tile_addr(tm.x_q, tm.x_col, tm.x_dig, ext_b, tbase, text, k0, &n_el);
                        int kk, r0;
                        entry(kc, t, kk, r0);
                        CHECK(kk < kc && r0 < RS, "entry decomposition");
                        const int d0 = r0 & 3, h = r0 >> 2;
                        if (kk >= kn || d0 >= ta.rem[0]) continue;
                        for (int it = 0; it < NIT; ++it) {
                            const int dd1 = RS == 8 ? 2 * (it & 1) : 0, d2 = RS == 8 ? it >> 1 : it;
                            if (!(h + dd1 < ta.rem[1] && d2 < ta.rem[2])) continue;
                            const int r = r0 + it * RS;
                            CHECK(r < R, "staged row %d beyond R", r);
                            // the entry holds digits (d0, h + dd1, d2) of row r
                            CHECK((r & 3) == d0 && ((r >> 2) & 3) == h + dd1 && (r >> 4) == d2, "entry digits");
                            const int64_t off = (int64_t)ta.base + (int64_t)kk * ta.sd + (int64_t)d0 * ta.s[0] +
                                                (int64_t)(h + dd1) * ta.s[1] + (int64_t)d2 * ta.s[2];
                            CHECK(off >= 0 && off < n_el, "global read outside the operand (term %d side %d)", p, side);
                        }
                    }
                }
            }
            // energy: eps reads of the thread's fixed labels and its owned 4 x 4
            if (fixed_ok) {
                for (int j = 0; j < 4; ++j) CHECK(tbase[a.fixed[j]] + f[j] < text[a.fixed[j]], "eps (fixed)");
                for (int o = 0; o < 2; ++o)
                    for (int u = 0; u < 4; ++u)
                        if (tbase[a.own[o]] + u < text[a.own[o]]) CHECK(tbase[a.own[o]] + u >= 0, "eps (owned)");
            }
        }
    }
}

// ---- FP32 kernel ----------------------------------------------------------------------------
static int deposit3(int v, int m) {
    int r = 0, b = 0;
    for (int j = 0; j < 6; ++j)
        if ((m >> j) & 1) { if ((v >> b) & 1) r |= 1 << j; ++b; }
    return r;
}
static int extract6(int t, int m) {
    int r = 0, b = 0;
    for (int j = 0; j < 6; ++j)
        if ((m >> j) & 1) { r |= ((t >> j) & 1) << b; ++b; }
    return r;
}
static int row_coord(int r, int i) { return 2 * ((r >> (3 + i)) & 1) + ((r >> i) & 1); }

struct SA { int base, sd, s[3], rem[3]; int64_t n_elems; };

// the kernel's stage_addr(), with the element count of the operand
static SA stage_addr(const int8_t *q, const int8_t *col, const int8_t *rank, const int32_t *ext_b, const int *tbase,
                     const int *text) {
    SA sa{};
    int st = 1;
    for (int m = 0; m < 4; ++m) {
        if (q[m] < 0) sa.sd = st;
        else {
            const int b0 = tbase[q[m]];
            sa.base += b0 * st;
            CHECK(rank[m] >= 0 && rank[m] < 3, "rank of a T label");
            sa.s[rank[m]] = st;
            sa.rem[rank[m]] = std::min(TS, text[q[m]] - b0);
        }
        st *= ext_b[col[m]];
    }
    sa.n_elems = st;
    return sa;
}

// element offset of an operand entry from the T coordinates (absolute) and the summed index
static int64_t direct_offset(const int8_t *q, const int8_t *col, const int32_t *ext_b, const int *coord, int k) {
    int64_t off = 0, st = 1;
    for (int m = 0; m < 4; ++m) {
        off += (int64_t)(q[m] < 0 ? k : coord[q[m]]) * st;
        st *= ext_b[col[m]];
    }
    return off;
}

static void replay32(const Args &a, const int32_t *ext_b) {
    static_assert(NT32 == 64 && ROW32 == 64 && RP32 >= ROW32 && (RP32 * 4) % 16 == 0, "FP32 kernel geometry");
    int text[6], ntile[6];
    for (int q = 0; q < 6; ++q) {
        text[q] = ext_b[a.t_col[q]];
        ntile[q] = (text[q] + TS - 1) / TS;
    }
    for (int mask = 0; mask < 64; ++mask) {
        int tbase[6];
        for (int q = 0; q < 6; ++q) tbase[q] = ((mask >> q) & 1) ? (ntile[q] - 1) * TS : 0;
        for (int p = 0; p < a.n_terms; ++p) {
            const TermDev &tm = a.term[p];
            const int K = ext_b[tm.d_col];
            const int M = tm.xmask;
            int pc = 0;
            for (int j = 0; j < 6; ++j) pc += (M >> j) & 1;
            CHECK(pc == 3 && (M & ~63) == 0, "X mask of term %d", p);
            // the 64 (x, y) pairs cover the 64 elements once
            std::vector<int> cnt(64, 0);
            for (int xi = 0; xi < 8; ++xi)
                for (int yi = 0; yi < 8; ++yi) ++cnt[deposit3(xi, M) | deposit3(yi, 63 & ~M)];
            for (int e = 0; e < 64; ++e) CHECK(cnt[e] == 1, "element %d covered %d times (term %d)", e, cnt[e], p);
            // packed pairs: the operand holding T label 0 gives entries (2m, 2m + 1) of its run;
            // with the other operand's entry bi they feed accumulator pair (e, e + 1), e even
            {
                const int MP = (M & 1) ? M : 63 & ~M;
                for (int m = 0; m < 4; ++m)
                    for (int bi = 0; bi < 8; ++bi) {
                        const int lo = deposit3(2 * m, MP) | deposit3(bi, 63 & ~MP);
                        const int hi = deposit3(2 * m + 1, MP) | deposit3(bi, 63 & ~MP);
                        CHECK((lo & 1) == 0 && hi == lo + 1, "packed pair (term %d, m %d, b %d)", p, m, bi);
                    }
            }
            SA sa[2];
            sa[0] = stage_addr(tm.x_q, tm.x_col, tm.x_rank, ext_b, tbase, text);
            sa[1] = stage_addr(tm.y_q, tm.y_col, tm.y_rank, ext_b, tbase, text);
            for (int k0 = 0; k0 < K; k0 += KC32) {
                const int kn = std::min(KC32, K - k0);
                // staging, as stage32 does it: thread r copies row r for kk < kn
                bool staged[2][ROW32];
                int64_t soff[2][ROW32];
                for (int side = 0; side < 2; ++side) {
                    const SA &x = sa[side];
                    const int8_t *q = side ? tm.y_q : tm.x_q, *col = side ? tm.y_col : tm.x_col;
                    for (int r = 0; r < NT32; ++r) {
                        const int c0 = row_coord(r, 0), c1 = row_coord(r, 1), c2 = row_coord(r, 2);
                        staged[side][r] = c0 < x.rem[0] && c1 < x.rem[1] && c2 < x.rem[2];
                        soff[side][r] = (int64_t)x.base + (int64_t)k0 * x.sd + (int64_t)c0 * x.s[0] +
                                        (int64_t)c1 * x.s[1] + (int64_t)c2 * x.s[2];
                        if (!staged[side][r]) continue;
                        CHECK(r < ROW32 && kn <= KC32 && (int64_t)(kn - 1) * RP32 + r < (int64_t)KC32 * RP32,
                              "shared entry beyond the tile");
                        int coord[6] = {0, 0, 0, 0, 0, 0};
                        for (int m = 0; m < 4; ++m)
                            if (q[m] >= 0) {
                                const int rk = (side ? tm.y_rank : tm.x_rank)[m];
                                coord[q[m]] = tbase[q[m]] + row_coord(r, rk);
                            }
                        for (int kk = 0; kk < kn; ++kk) {
                            const int64_t g = soff[side][r] + (int64_t)kk * x.sd;
                            CHECK(g >= 0 && g < x.n_elems, "global read outside the operand (term %d side %d)", p, side);
                            CHECK(g == direct_offset(q, col, ext_b, coord, k0 + kk),
                                  "entry (%d, %d) staged from the wrong element (term %d side %d)", kk, r, p, side);
                        }
                    }
                }
                // products: every element inside the block reads the entries at its coordinates
                for (int t = 0; t < NT32; ++t) {
                    bool live = true;
                    for (int j = 0; j < 6; ++j) live &= tbase[j] + 2 * ((t >> j) & 1) < text[j];
                    if (!live) continue;
                    const int hx = extract6(t, M), hy = extract6(t, 63 & ~M);
                    // the operand holding T label 0 is read from P, the other one from B (8
                    // entries at 8 h each)
                    const int MP = (M & 1) ? M : 63 & ~M;
                    const int hp = extract6(t, MP), hb = extract6(t, 63 & ~MP);
                    CHECK((8 * hp * 4) % 16 == 0 && (RP32 * 4) % 16 == 0 &&
                          (int64_t)(kn - 1) * RP32 + 8 * hp + 8 <= (int64_t)KC32 * RP32, "P loads of thread %d", t);
                    CHECK((8 * hb * 4) % 16 == 0 &&
                          (int64_t)(kn - 1) * RP32 + 8 * hb + 8 <= (int64_t)KC32 * RP32, "B loads of thread %d", t);
                    CHECK(hp == ((M & 1) ? hx : hy) && hb == ((M & 1) ? hy : hx), "operand groups of thread %d", t);
                    for (int xi = 0; xi < 8; ++xi)
                        for (int yi = 0; yi < 8; ++yi) {
                            const int e = deposit3(xi, M) | deposit3(yi, 63 & ~M);
                            int coord[6];
                            bool in = true;
                            for (int j = 0; j < 6; ++j) {
                                coord[j] = tbase[j] + 2 * ((t >> j) & 1) + ((e >> j) & 1);
                                in &= coord[j] < text[j];
                            }
                            if (!in) continue;
                            for (int side = 0; side < 2; ++side) {
                                const int row = side ? 8 * hy + yi : 8 * hx + xi;
                                CHECK(staged[side][row], "element reads an unstaged row (term %d side %d)", p, side);
                                const int64_t want = direct_offset(side ? tm.y_q : tm.x_q, side ? tm.y_col : tm.x_col,
                                                                   ext_b, coord, k0);
                                CHECK(soff[side][row] == want, "row %d holds the wrong entry (term %d side %d)", row, p,
                                      side);
                            }
                        }
                }
            }
        }
        // energy: eps reads at coordinates inside the block
        for (int t = 0; t < NT32; ++t)
            for (int j = 0; j < 6; ++j)
                for (int l = 0; l < 2; ++l) {
                    const int c = tbase[j] + 2 * ((t >> j) & 1) + l;
                    if (c < text[j]) CHECK(c >= 0, "eps read");
                }
    }
}

// ---- FP32 tensor-core path (k_triples_tc.cu) --------------------------------------------------
// the kernels' op_geo(): the operand's T labels in T order with strides, extents, tile sizes and
// counts; the summed label's stride and extent
struct Geo { int lab[3], st[3], ext[3], ts[3], nt[3], sd, ed, nch, rpt; bool wide; };

static Geo op_geo(const TermDev &tm, int side, const int32_t *ext_b) {
    const int8_t *q = side ? tm.y_q : tm.x_q, *col = side ? tm.y_col : tm.x_col, *rk = side ? tm.y_rank : tm.x_rank;
    Geo g{};
    int st = 1;
    for (int m = 0; m < 4; ++m) {
        const int e = ext_b[col[m]];
        if (q[m] < 0) g.sd = st;
        else { g.lab[rk[m]] = q[m]; g.st[rk[m]] = st; g.ext[rk[m]] = e; }
        st *= e;
    }
    g.ed = ext_b[tm.d_col];
    g.nch = (g.ed + tc::KCH - 1) / tc::KCH;
    g.wide = g.lab[0] == 0;
    g.rpt = g.wide ? tc::WROWS : tc::NROWS;
    for (int i = 0; i < 3; ++i) {
        g.ts[i] = g.lab[i] == 0 ? tc::WA : TS;
        g.nt[i] = (g.ext[i] + g.ts[i] - 1) / g.ts[i];
    }
    return g;
}
static void tc_row_coords(bool wide, int r, int &c0, int &c1, int &c2) {
    if (wide) { c0 = r & 7; c1 = (r >> 3) & 3; c2 = r >> 5; }
    else { c0 = r & 3; c1 = (r >> 2) & 3; c2 = r >> 4; }
}

static void replay_tc(const Plan &P, const Args &a) {
    const TriplesPlan &tp = P.tri;
    CHECK(!tp.tc_batch.empty(), "FP32 plan without the tensor-core layout");
    if (tp.tc_batch.empty()) return;
    // the pair-tile in shared memory: one slot per element, inside TSZ; the 32 rows a drain warp
    // holds (8 along label 0 x 4 along label L) fall in 32 different banks
    {
        std::vector<int> seen(tc::TSZ, 0);
        for (int e = 0; e < 8 * 1024; ++e) {
            const int c[6] = {e & 7, (e >> 3) & 3, (e >> 5) & 3, (e >> 7) & 3, (e >> 9) & 3, (e >> 11) & 3};
            int off = 0;
            for (int q = 0; q < 6; ++q) off += tc::tstride(q) * c[q];
            CHECK(off >= 0 && off < tc::TSZ, "pair-tile offset outside TSZ");
            if (off >= 0 && off < tc::TSZ) ++seen[off];
        }
        int twice = 0;
        for (int v : seen) twice += v > 1;
        CHECK(twice == 0, "pair-tile slots shared by %d elements", twice);
        for (int L = 1; L < 6; ++L) {
            int banks = 0;
            for (int c0 = 0; c0 < 8; ++c0)
                for (int c1 = 0; c1 < 4; ++c1) banks |= 1 << ((c0 + tc::tstride(L) * c1) & 31);
            CHECK(banks == -1, "drain rows of label %d share banks", L);
        }
    }
    const int nb = tp.n_blocks, nt = tp.n_terms;
    CHECK(tp.tc_batch.front() == 0 && tp.tc_batch.back() == nb, "batches cover the blocks");
    for (size_t bi = 0; bi + 1 < tp.tc_batch.size(); ++bi) {
        int64_t next = 0;   // operands of a batch are consecutive from row 0
        for (int b = tp.tc_batch[bi]; b < tp.tc_batch[bi + 1]; ++b) {
            const int32_t *ext_b = tp.ext.data() + (size_t)b * tp.n_labels;
            for (int p = 0; p < nt; ++p)
                for (int side = 0; side < 2; ++side) {
                    const Geo g = op_geo(a.term[p], side, ext_b);
                    const int64_t rows = (int64_t)g.nt[0] * g.nt[1] * g.nt[2] * g.nch * 3 * g.rpt;
                    const int64_t r0 = tp.tc_row0[((size_t)b * nt + p) * 2 + side];
                    CHECK(r0 == next, "operand (%d, %d, %d) does not follow the previous one", b, p, side);
                    next = r0 + rows;
                    CHECK(next <= tp.tc_max_rows && next < (int64_t(1) << 31), "operand beyond the batch region");
                }
        }
    }
    for (int b = 0; b < nb; ++b) {
        const int32_t *ext_b = tp.ext.data() + (size_t)b * tp.n_labels;
        int text[6], ntile[6];
        int64_t items = 1;
        for (int q = 0; q < 6; ++q) {
            text[q] = ext_b[a.t_col[q]];
            ntile[q] = (text[q] + (q == 0 ? tc::WA : TS) - 1) / (q == 0 ? tc::WA : TS);
            items *= ntile[q];
        }
        CHECK(tp.tc_prefix[b + 1] - tp.tc_prefix[b] == items, "pair-tiles of block %d", b);
        // pair-tiles: the first and the last along every label
        for (int mask = 0; mask < 64; ++mask) {
            int tcq[6], tbase[6];
            for (int q = 0; q < 6; ++q) {
                tcq[q] = ((mask >> q) & 1) ? ntile[q] - 1 : 0;
                tbase[q] = tcq[q] * (q == 0 ? tc::WA : TS);
            }
            // the kernels' decode of this item's linear index gives back these coordinates
            int64_t lin = 0;
            for (int q = 5; q >= 0; --q) lin = lin * ntile[q] + tcq[q];
            {
                int64_t rem = lin;
                for (int q = 0; q < 6; ++q) {
                    const int64_t qt = rem / ntile[q];
                    CHECK((int)(rem - qt * ntile[q]) == tcq[q], "item decode");
                    rem = qt;
                }
            }
            for (int p = 0; p < nt; ++p) {
                const TermDev &tm = a.term[p];
                const int sw = (tm.xmask & 1) ? 0 : 1;
                const Geo gs[2] = {op_geo(tm, sw, ext_b), op_geo(tm, 1 - sw, ext_b)};   // wide, narrow
                CHECK(gs[0].wide && !gs[1].wide, "term %d: the operand holding label 0", p);
                int64_t orow[2];
                for (int w = 0; w < 2; ++w) {
                    const Geo &g = gs[w];
                    const int side = w == 0 ? sw : 1 - sw;
                    const int64_t r0 = tp.tc_row0[((size_t)b * nt + p) * 2 + side];
                    const int64_t tile = tcq[g.lab[0]] + (int64_t)g.nt[0] * (tcq[g.lab[1]] + (int64_t)g.nt[1] * tcq[g.lab[2]]);
                    orow[w] = r0 + tile * g.nch * 3 * g.rpt;
                    const int64_t seg_end = r0 + (int64_t)g.nt[0] * g.nt[1] * g.nt[2] * g.nch * 3 * g.rpt;
                    // the producer's boxes: 64 rows at row + (ch * 3 + plane) * rows per tile (+ 64)
                    for (int ch = 0; ch < g.nch; ++ch)
                        for (int pl = 0; pl < 3; ++pl)
                            for (int h = 0; h < g.rpt / tc::BOX; ++h) {
                                const int64_t br = orow[w] + ((int64_t)ch * 3 + pl) * g.rpt + h * tc::BOX;
                                CHECK(br >= r0 && br + tc::BOX <= seg_end, "box outside operand (term %d)", p);
                            }
                }
                // the host-built term record gives the same rows as a linear form in the tile
                // coordinates
                {
                    TcRec rec;
                    std::memcpy(&rec, tp.tc_rec.data() + ((size_t)b * nt + p) * 16, sizeof(rec));
                    for (int w = 0; w < 2; ++w) {
                        int64_t v = rec.row0[w];
                        for (int q = 0; q < 6; ++q) v += (int64_t)rec.coef[w][q] * tcq[q];
                        CHECK(v == orow[w], "term %d: record row of operand %d", p, w);
                    }
                    CHECK(rec.nch == gs[0].nch && rec.ed == gs[0].ed, "term %d: record chunks", p);
                }
                // the drain's index map against the elements' coordinates (warp columns 16 colq + j,
                // j = c0 + 4 c1, at the narrow labels' coordinates (c0, c1, colq)), and the pre-pass's
                // rows against the operand elements at those coordinates
                int lw[3] = {gs[0].lab[0], gs[0].lab[1], gs[0].lab[2]}, ln[3] = {gs[1].lab[0], gs[1].lab[1], gs[1].lab[2]};
                std::vector<int> hit(tc::TSZ, 0);
                for (int m = 0; m < tc::WROWS; ++m) {
                    const int offw = (m & 7) + tc::tstride(lw[1]) * ((m >> 3) & 3) + tc::tstride(lw[2]) * (m >> 5);
                    for (int n = 0; n < tc::NROWS; ++n) {
                        const int off = offw + tc::tstride(ln[0]) * (n & 3) + tc::tstride(ln[1]) * ((n >> 2) & 3) +
                                        tc::tstride(ln[2]) * (n >> 4);
                        int cin[6];
                        int wc[3], nc[3];
                        tc_row_coords(true, m, wc[0], wc[1], wc[2]);
                        tc_row_coords(false, n, nc[0], nc[1], nc[2]);
                        for (int i = 0; i < 3; ++i) { cin[lw[i]] = wc[i]; cin[ln[i]] = nc[i]; }
                        int want = 0;
                        for (int q = 0; q < 6; ++q) want += tc::tstride(q) * cin[q];
                        CHECK(off == want, "term %d: (%d, %d) drained to the wrong element", p, m, n);
                        if (off >= 0 && off < tc::TSZ) ++hit[off];
                    }
                }
                int cover = 0;
                for (int v : hit) cover += v == 1;
                CHECK(cover == 8192, "term %d covers %d pair-tile elements once", p, cover);
                // rows of the wide and narrow tiles hold the operand at the element coordinates
                for (int w = 0; w < 2; ++w) {
                    const Geo &g = gs[w];
                    const int side = w == 0 ? sw : 1 - sw;
                    const int8_t *q = side ? tm.y_q : tm.x_q, *col = side ? tm.y_col : tm.x_col;
                    const int64_t r0 = tp.tc_row0[((size_t)b * nt + p) * 2 + side];
                    for (int r = 0; r < g.rpt; ++r) {
                        int c[3];
                        tc_row_coords(g.wide, r, c[0], c[1], c[2]);
                        // the pre-pass's view of this plane row: R = tile * rpt + r
                        const int64_t tile = (orow[w] - r0) / (g.nch * 3 * g.rpt);
                        const int t0 = (int)(tile % g.nt[0]), t1 = (int)((tile / g.nt[0]) % g.nt[1]),
                                  t2 = (int)(tile / ((int64_t)g.nt[0] * g.nt[1]));
                        const int gg[3] = {t0 * g.ts[0] + c[0], t1 * g.ts[1] + c[1], t2 * g.ts[2] + c[2]};
                        bool valid = true;
                        int coord[6] = {0, 0, 0, 0, 0, 0};
                        for (int i = 0; i < 3; ++i) {
                            valid &= gg[i] < g.ext[i];
                            CHECK(gg[i] == tbase[g.lab[i]] + c[i], "plane row %d of term %d at the wrong tile", r, p);
                            coord[g.lab[i]] = gg[i];
                        }
                        if (!valid) continue;
                        for (int k = 0; k < g.ed; k += std::max(1, g.ed - 1)) {
                            const int64_t ro = (int64_t)gg[0] * g.st[0] + (int64_t)gg[1] * g.st[1] + (int64_t)gg[2] * g.st[2] +
                                               (int64_t)k * g.sd;
                            CHECK(ro == direct_offset(q, col, ext_b, coord, k), "pre-pass row %d reads the wrong element", r);
                        }
                    }
                }
            }
            // energy: thread et takes labels 0..3 at (et & 7, et >> 3 & 3, et >> 5 & 3, et >> 7) and
            // labels 4, 5 at (u & 3, u >> 2): each element once
            static_assert(32 * tc::DRAIN_WARPS == 512, "one energy thread per labels 0..3 combination");
            std::vector<int> eh(tc::TSZ, 0);
            for (int et = 0; et < 32 * tc::DRAIN_WARPS; ++et)
                for (int u = 0; u < 16; ++u) {
                    const int cj = u & 3, ck = u >> 2;
                    const int off = (et & 7) + tc::tstride(1) * ((et >> 3) & 3) + tc::tstride(2) * ((et >> 5) & 3) +
                                    tc::tstride(3) * ((et >> 7) & 3) + tc::tstride(4) * cj + tc::tstride(5) * ck;
                    CHECK(off < tc::TSZ, "energy read outside the pair-tile");
                    if (off < tc::TSZ) ++eh[off];
                }
            int once = 0;
            for (int v : eh) once += v == 1;
            CHECK(once == 8192, "energy reads %d elements once", once);
        }
    }
}

// the kernels' ItemWalk (mixed-radix advance of the tile coordinates by the grid stride, forward
// block scan) against a direct decode of every item index, on blocks of random extents (many with
// fewer pair-tiles than the stride) and several strides
static void replay_item_walk() {
    uint64_t st = 88172645463325252ull;
    auto rnd = [&](int lo, int hi) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        return lo + (int)(st % (uint64_t)(hi - lo + 1));
    };
    const int nb = 200;
    std::vector<std::array<int, 6>> rad(nb);
    std::vector<int64_t> prefix(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        int64_t c = 1;
        for (int q = 0; q < 6; ++q) {
            const int e = rnd(1, b % 3 == 0 ? 3 : 20);
            const int ts = q == 0 ? tc::WA : TS;
            rad[b][q] = (e + ts - 1) / ts;
            c *= rad[b][q];
        }
        prefix[b + 1] = prefix[b] + c;
    }
    for (int stride : {1, 7, 152, 1000}) {
        for (int first = 0; first < std::min(stride, 3); ++first) {
            // the walk, as the kernels run it
            int b = 0, tc[6] = {0, 0, 0, 0, 0, 0}, step[6] = {0, 0, 0, 0, 0, 0};
            uint32_t local = 0, count = 0;
            int64_t g = first;
            auto enter = [&]() {
                uint32_t rem = local, s2 = (uint32_t)stride;
                for (int q = 0; q < 6; ++q) {
                    const uint32_t n = (uint32_t)rad[b][q];
                    tc[q] = (int)(rem % n); rem /= n;
                    step[q] = (int)(s2 % n); s2 /= n;
                }
                count = (uint32_t)(prefix[b + 1] - prefix[b]);
            };
            auto locate = [&](int from) {
                b = from;
                while (b + 1 < nb && prefix[b + 1] <= g) ++b;
                local = (uint32_t)(g - prefix[b]);
                enter();
            };
            locate(0);
            for (; g < prefix[nb];) {
                // direct decode
                int db = 0;
                while (prefix[db + 1] <= g) ++db;
                int64_t rem = g - prefix[db];
                bool same = db == b;
                for (int q = 0; q < 6; ++q) { same &= (int)(rem % rad[db][q]) == tc[q]; rem /= rad[db][q]; }
                CHECK(same, "item walk at item %lld (stride %d)", (long long)g, stride);
                g += stride;
                if (g >= prefix[nb]) break;
                local += (uint32_t)stride;
                if (local < count) {
                    int carry = 0;
                    for (int q = 0; q < 6; ++q) {
                        const int d = tc[q] + step[q] + carry;
                        carry = d >= rad[b][q];
                        tc[q] = carry ? d - rad[b][q] : d;
                    }
                } else {
                    locate(b);
                }
            }
        }
    }
}

int main(int argc, char **argv) {
    if (argc < 2) { std::printf("usage\n"); return 2; }
    const int nt = std::atoi(argv[1]);
    if (argc != 2 + nt + 7 + 6 + 7) { std::printf("bad arguments\n"); return 2; }
    std::vector<const char *> terms(argv + 2, argv + 2 + nt);
    const char *names[7];
    for (int l = 0; l < 7; ++l) names[l] = argv[2 + nt + l];
    int signs[6];
    for (int q = 0; q < 6; ++q) signs[q] = std::atoi(argv[2 + nt + 7 + q]);
    int64_t ext[7];
    for (int l = 0; l < 7; ++l) ext[l] = std::atoll(argv[2 + nt + 13 + l]);
    for (int e : {4, 8}) {
        Plan P;
        std::string err;
        comet_status_t st = plan_triples(terms.data(), nt, names, 7, 1, ext, signs, e == 4 ? COMET_F32 : COMET_F64,
                                         &P, &err);
        CHECK(st == COMET_OK, "plan: %s", err.c_str());
        if (st != COMET_OK) continue;
        Args a;
        std::memset(&a, 0, sizeof(a));
        triples_args(P, &a);
        if (e == 4) {
            replay32(a, P.tri.ext.data());
            replay_tc(P, a);
        } else {
            replay(a, P.tri.ext.data(), e);
        }
    }
    replay_item_walk();
    std::printf("%d failures\n", fails);
    return fails ? 1 : 0;
}
