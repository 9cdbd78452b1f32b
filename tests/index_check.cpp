// CPU replay of the transpose engine's index arithmetic (the loop nests of xpose_tile_kernel
// and xpose_copy_kernel) over many random shapes, permutations and strided outputs, and of
// the GEMM offset groups.  Checks that every access stays inside its buffer, that vector
// accesses are aligned, and that every output element is written exactly once from the
// right input element.  Built and run by tests/test_index_check.py; exit status 0 = pass.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2102_06827_gb300/csrc/plan.hpp"

using namespace comet;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

// replay of xpose_tile_kernel / xpose_copy_kernel: fills the output->input map
// in_off / out_off: element offsets of the first element (views) from 16-byte aligned bases;
// n_in / n_out_span and src_of_out count from the bases
static bool replay(const XposeParams &p, int vi, int vo, int64_t n_in, int64_t n_out_span,
                   std::vector<int64_t> &src_of_out, int64_t in_off = 0, int64_t out_off = 0) {
    const int XT = 256, XTAB = 256;
    const bool copy = vo < 0;
    CHECK(p.tu >= 1 && p.tv >= 1 && p.tw >= 1, "empty tile");
    CHECK((uint64_t)p.tu * p.tv * p.tw <= 8192 + 3 * 256 || (copy && p.tv == 1 && p.tw == 1), "tile too large");
    CHECK(copy || xpose_smem_bytes(p, 8) <= 96 * 1024, "tile exceeds the shared memory it is given");
    CHECK(p.tv <= (uint32_t)XTAB && p.tw <= (uint32_t)XTAB, "tile edge above the table size");
    CHECK(copy || p.tu <= (uint32_t)XTAB, "transposing tile edge above the table size");
    CHECK(p.ll >= 1 && p.sl >= 1 && p.sl <= (uint32_t)XT, "lane counts");
    CHECK(p.rpp_s == (uint32_t)XT / p.sl && (p.ll > (uint32_t)XT || p.rpp_l == (uint32_t)XT / p.ll), "rows per pass");
    CHECK(copy || p.ll <= (uint32_t)XT, "load lanes above the block");
    CHECK(p.ll == (p.tu + (uint32_t)(copy ? -vo : vi) - 1) / (uint32_t)(copy ? -vo : vi), "load lanes vs vector width");
    CHECK(copy || p.sl == (p.tv + (uint32_t)vo - 1) / (uint32_t)vo, "store lanes vs vector width");
    CHECK(vi == 1 || vi * 4 == 16 || vi * 8 == 16, "vector width");
    const uint64_t grid = (uint64_t)p.tiles_u * p.tiles_v * p.tiles_w;
    const uint32_t tu = p.tu, tv = p.tv, tw = p.tw, pitch = tu | 1u;
    const int64_t su = p.u.s0[0];
    {   // U is affine in the input with stride su (and, in copy mode, in the output with p.u.s1[0])
        int64_t s = su;
        for (int d = 0; d < p.u.n; ++d) { CHECK(p.u.s0[d] == s, "U not affine in the input"); s *= p.u.ext[d]; }
        CHECK(!copy || p.u.n <= 1, "copy-mode U with several digits");
    }
    if (!copy) {   // V is affine in the output with stride sv
        int64_t s = p.v.s1[0];
        for (int d = 0; d < p.v.n; ++d) { CHECK(p.v.s1[d] == s, "V not affine in the output"); s *= p.v.ext[d]; }
    }
    for (uint64_t blk = 0; blk < grid && fails == 0; ++blk) {
        if (copy) {
            const uint32_t bw = fd_div((uint32_t)blk, p.fd_tiles_u), bu = (uint32_t)blk - bw * p.tiles_u;
            CHECK(bu == blk % p.tiles_u && bw == blk / p.tiles_u, "block decomposition");
            const uint32_t u0 = bu * tu, w0 = bw * tw;
            const uint32_t nu = std::min(tu, p.u.total - u0), nw = std::min(tw, p.r.total - w0);
            const int64_t so = p.u.s1[0];
            const int VW = -vo;
            std::vector<int64_t> row_in(nw), row_out(nw);
            CHECK(nw <= (uint32_t)XTAB, "rows above the table size");
            for (uint32_t i = 0; i < nw; ++i) {
                int64_t a, c;
                radix_offsets(p.r, w0 + i, a, c);
                row_in[i] = a + (int64_t)u0 * su;
                row_out[i] = c + (int64_t)u0 * so;
                CHECK(!p.off32 || (row_in[i] < (1ll << 31) && row_out[i] < (1ll << 31)), "32-bit row offset overflows");
            }
            auto move = [&](uint32_t u, uint32_t row) {
                const int64_t si = in_off + row_in[row] + (int64_t)u * su, d = out_off + row_out[row] + (int64_t)u * so;
                CHECK(si % VW == 0 && d % VW == 0, "misaligned copy vector");
                for (int q = 0; q < VW; ++q) {
                    CHECK(u + q < nu, "vector crosses the tile");
                    CHECK(VW == 1 || (su == 1 && so == 1), "vector along a strided run");
                    const int64_t a = si + q * su, c = d + q * so;
                    CHECK(a >= 0 && a < n_in && c >= 0 && c < n_out_span, "copy out of bounds");
                    if (c >= 0 && c < n_out_span) { CHECK(src_of_out[c] == -1, "written twice"); src_of_out[c] = a; }
                }
            };
            CHECK(VW > 2 || (uint64_t)tu * tw * 8 <= 48 * 1024, "copy-mode stage above 48 KB of shared memory");
            const uint32_t lanes = p.ll;
            if (p.single_run) {
                CHECK(nw == 1 && p.r.total == 1, "long-row copy with several rows");
                CHECK(p.tiles_u == 1 || tu % VW == 0, "long-row tiles do not start on a vector boundary");
                const uint32_t nvec = nu / VW * VW;
                for (uint32_t t = 0; t < (uint32_t)XT; ++t)
                    for (uint32_t u = t * VW; u < nvec; u += XT * VW) move(u, 0);
                CHECK(nu - nvec <= (uint32_t)XT, "tail longer than the block");
                for (uint32_t t = 0; t < nu - nvec; ++t) {   // element-wise tail
                    const uint32_t u = nvec + t;
                    const int64_t a = in_off + row_in[0] + (int64_t)u * su, c = out_off + row_out[0] + (int64_t)u * so;
                    CHECK(a >= 0 && a < n_in && c >= 0 && c < n_out_span, "tail out of bounds");
                    if (c >= 0 && c < n_out_span) { CHECK(src_of_out[c] == -1, "written twice"); src_of_out[c] = a; }
                }
                continue;
            }
            CHECK(lanes <= (uint32_t)XT, "row copy with more lanes than threads");
            const uint32_t rpp = p.rpp_l;
            for (uint32_t t = 0; t < (uint32_t)XT; ++t) {
                const uint32_t r0 = fd_div(t, p.fd_ll), u = (t - r0 * lanes) * VW;
                if (!(r0 < rpp && u < nu)) continue;
                for (uint32_t row = r0; row < nw; row += rpp) move(u, row);
            }
            continue;
        }
        const uint32_t b = fd_div((uint32_t)blk, p.fd_tiles_u), bu = (uint32_t)blk - b * p.tiles_u;
        const uint32_t bw = fd_div(b, p.fd_tiles_v), bv = b - bw * p.tiles_v;
        CHECK(bu == blk % p.tiles_u && bv == (blk / p.tiles_u) % p.tiles_v && bw == blk / p.tiles_u / p.tiles_v, "block decomposition");
        const uint32_t u0 = bu * tu, v0 = bv * tv, w0 = bw * tw;
        const uint32_t nu = std::min(tu, p.u.total - u0), nv = std::min(tv, p.v.total - v0),
                       nw = std::min(tw, p.r.total - w0);
        const int64_t sv = p.v.s1[0];
        std::vector<int64_t> uo(nu), vin(nv), win(nw), wout(nw);
        for (uint32_t i = 0; i < nu; ++i) { int64_t a; radix_offsets(p.u, u0 + i, a, uo[i]); CHECK(a == (int64_t)(u0 + i) * su, "U input offset"); }
        for (uint32_t i = 0; i < nv; ++i) { int64_t c; radix_offsets(p.v, v0 + i, vin[i], c); CHECK(c == (int64_t)(v0 + i) * sv, "V output offset"); }
        for (uint32_t i = 0; i < nw; ++i) radix_offsets(p.r, w0 + i, win[i], wout[i]);
        const uint32_t rows_v = nv * nw, rows_u = nu * nw;
        std::vector<int64_t> in_row(rows_v), out_o(rows_u), out_s(rows_u);
        for (uint32_t r = 0; r < rows_v; ++r) {
            uint32_t w = nv == tv ? fd_div(r, p.fd_tv) : r / nv, v = r - w * nv;
            CHECK(w == r / nv, "row division (v)");
            in_row[r] = (int64_t)u0 * su + vin[v] + win[w];
        }
        for (uint32_t r = 0; r < rows_u; ++r) {
            uint32_t w = nu == tu ? fd_div(r, p.fd_tu) : r / nu, u = r - w * nu;
            CHECK(w == r / nu, "row division (u)");
            out_o[r] = (int64_t)v0 * sv + uo[u] + wout[w];
            out_s[r] = (int64_t)w * nv * pitch + u;
        }
        for (uint32_t r = 0; r < rows_v; ++r) CHECK(!p.off32 || in_row[r] < (1ll << 31), "32-bit input row offset overflows");
        for (uint32_t r = 0; r < rows_u; ++r) CHECK(!p.off32 || out_o[r] < (1ll << 31), "32-bit output row offset overflows");
        std::vector<int64_t> buf((size_t)tw * tv * pitch, -1);
        {   // loads: p.ll threads per row, fixed u, rows (v, w) walked
            const uint32_t lanes = p.ll, rpp = p.rpp_l;
            CHECK(rpp >= 1, "no rows per pass (load)");
            for (uint32_t t = 0; t < (uint32_t)XT; ++t) {
                const uint32_t r0 = fd_div(t, p.fd_ll), u = (t - r0 * lanes) * vi;
                if (!(r0 < rpp && u < nu)) continue;
                for (uint32_t row = r0; row < rows_v; row += rpp) {
                    const int64_t src = in_off + (int64_t)u * su + in_row[row];
                    CHECK(src % vi == 0, "misaligned vector load");
                    for (int q = 0; q < vi; ++q) {
                        CHECK(u + q < nu, "vector load crosses the tile");
                        CHECK(vi == 1 || su == 1, "vector load along a strided run");
                        CHECK(src + q >= 0 && src + q < n_in, "load out of bounds");
                        const size_t bi = (size_t)row * pitch + u + q;
                        CHECK(bi < buf.size(), "shared store out of the tile");
                        if (bi < buf.size()) buf[bi] = src + q;
                    }
                }
            }
        }
        {   // stores: p.sl threads per row, fixed v, rows (u, w) walked
            const uint32_t lanes = p.sl, rpp = p.rpp_s;
            CHECK(rpp >= 1, "no rows per pass (store)");
            for (uint32_t t = 0; t < (uint32_t)XT; ++t) {
                const uint32_t r0 = fd_div(t, p.fd_sl), v = (t - r0 * lanes) * vo;
                if (!(r0 < rpp && v < nv)) continue;
                for (uint32_t row = r0; row < rows_u; row += rpp) {
                    const int64_t dst = out_off + out_o[row] + (int64_t)v * sv;
                    CHECK(dst % vo == 0, "misaligned vector store");
                    for (int q = 0; q < vo; ++q) {
                        CHECK(v + q < nv, "vector store crosses the tile");
                        CHECK(vo == 1 || sv == 1, "vector store along a strided run");
                        const size_t bi = (size_t)(v + q) * pitch + out_s[row];
                        CHECK(bi < buf.size(), "shared load out of the tile");
                        const int64_t s2 = bi < buf.size() ? buf[bi] : -1;
                        CHECK(s2 >= 0, "store of an element that was not loaded");
                        const int64_t d = dst + q;
                        CHECK(d >= 0 && d < n_out_span, "store out of bounds");
                        if (d >= 0 && d < n_out_span) { CHECK(src_of_out[d] == -1, "written twice"); src_of_out[d] = s2; }
                    }
                }
            }
        }
    }
    return fails == 0;
}

int main() {
    std::mt19937_64 rng(12345);
    int cases = 0;
    // dense permutations (comet_transpose)
    for (int it = 0; it < 3000 && fails == 0; ++it) {
        int rank = 1 + rng() % 6;
        int64_t ext[8], si[8], so[8], so_out[8];
        int perm[8];
        int64_t n = 1;
        for (int d = 0; d < rank; ++d) {
            int pick = rng() % 10;
            ext[d] = pick < 2 ? 1 : pick < 5 ? 1 + rng() % 5 : pick < 8 ? 8 * (1 + rng() % 4) : 1 + rng() % 70;
            n *= ext[d];
        }
        if (n > 400000) continue;
        for (int d = 0; d < rank; ++d) perm[d] = d;
        std::shuffle(perm, perm + rank, rng);
        int64_t s = 1;
        for (int d = 0; d < rank; ++d) { si[d] = s; s *= ext[d]; }
        s = 1;
        for (int d = 0; d < rank; ++d) { so_out[d] = s; s *= ext[perm[d]]; }
        for (int d = 0; d < rank; ++d) so[perm[d]] = so_out[d];
        for (int es : {4, 8}) {
            XposeParams p;
            int vi, vo;
            double eff;
            setup_xpose(rank, ext, si, so, es, &p, &vi, &vo, &eff);
            std::vector<int64_t> map(n, -1);
            replay(p, vi, vo, n, n, map);
            // expected: out[j] = in[i] with i[perm[d]] = j_d
            for (int64_t j = 0; j < n && fails == 0; ++j) {
                int64_t rem = j, off = 0;
                for (int d = 0; d < rank; ++d) { off += (rem % ext[perm[d]]) * si[perm[d]]; rem /= ext[perm[d]]; }
                CHECK(map[j] == off, "rank %d case %d: out %lld from %lld, expected %lld", rank, it,
                      (long long)j, (long long)map[j], (long long)off);
            }
            ++cases;
        }
    }
    // fixed cases: long single fused runs (affine copy path), identity and near-identity
    // permutations, tiny leading extents on one or both sides
    {
        struct Fx { int rank; int64_t ext[6]; int perm[6]; };
        const Fx fx[] = {{1, {5000}, {0}}, {1, {4999}, {0}}, {1, {8193}, {0}}, {2, {257, 3}, {0, 1}}, {2, {300, 500}, {0, 1}}, {3, {54, 97, 7}, {0, 1, 2}},
                         {3, {9, 13, 100}, {1, 2, 0}}, {4, {9, 13, 10, 8}, {1, 0, 3, 2}},
                         {3, {2000, 9, 5}, {1, 0, 2}}, {2, {4096, 3}, {0, 1}}, {3, {300, 2, 5}, {0, 2, 1}},
                         {6, {8, 11, 5, 6, 13, 8}, {1, 2, 4, 5, 3, 0}}};
        for (const Fx &f : fx) {
            int64_t si[8], so[8], so_out[8], n = 1, s = 1;
            for (int d = 0; d < f.rank; ++d) { si[d] = s; s *= f.ext[d]; }
            n = s;
            s = 1;
            for (int d = 0; d < f.rank; ++d) { so_out[d] = s; s *= f.ext[f.perm[d]]; }
            for (int d = 0; d < f.rank; ++d) so[f.perm[d]] = so_out[d];
            for (int es : {4, 8}) {
                XposeParams p;
                int vi, vo;
                double eff;
                setup_xpose(f.rank, f.ext, si, so, es, &p, &vi, &vo, &eff);
                std::vector<int64_t> map(n, -1);
                replay(p, vi, vo, n, n, map);
                for (int64_t j = 0; j < n && fails == 0; ++j) {
                    int64_t rem = j, off = 0;
                    for (int d = 0; d < f.rank; ++d) { off += (rem % f.ext[f.perm[d]]) * si[f.perm[d]]; rem /= f.ext[f.perm[d]]; }
                    CHECK(map[j] == off, "fixed case rank %d: out %lld", f.rank, (long long)j);
                }
                ++cases;
            }
        }
    }
    // views: strided slices (lo, step) of stored tensors on both sides at element offsets that
    // need not be 16-byte aligned; every view element lands once, from the right element
    for (int it = 0; it < 3000 && fails == 0; ++it) {
        const int rank = 1 + rng() % 4;
        int64_t ext[8], decl_in[8], decl_out[8], lo_in[8], lo_out[8], st_in[8], st_out[8];
        int perm[8];
        int64_t n = 1;
        for (int d = 0; d < rank; ++d) {
            const int pick = rng() % 6;
            ext[d] = pick < 1 ? 1 : pick < 3 ? 1 + rng() % 9 : 4 * (1 + rng() % 12) + (pick == 5 ? 1 : 0);
            n *= ext[d];
        }
        if (n > 100000) continue;
        for (int d = 0; d < rank; ++d) perm[d] = d;
        std::shuffle(perm, perm + rank, rng);
        for (int d = 0; d < rank; ++d) {   // input dimension d, output dimension d (label perm[d])
            st_in[d] = rng() % 3 == 0 ? 1 + rng() % 3 : 1;
            lo_in[d] = rng() % 3;
            decl_in[d] = lo_in[d] + (ext[d] - 1) * st_in[d] + 1 + rng() % 3;
            st_out[d] = rng() % 3 == 0 ? 1 + rng() % 3 : 1;
            lo_out[d] = rng() % 3;
            decl_out[d] = lo_out[d] + (ext[perm[d]] - 1) * st_out[d] + 1 + rng() % 3;
        }
        int64_t si[8], so[8], S = 1, in_off = 0, out_off = 0, n_in = 1, n_out = 1;
        for (int d = 0; d < rank; ++d) { si[d] = st_in[d] * S; in_off += lo_in[d] * S; S *= decl_in[d]; }
        n_in = S;
        S = 1;
        for (int d = 0; d < rank; ++d) { so[perm[d]] = st_out[d] * S; out_off += lo_out[d] * S; S *= decl_out[d]; }
        n_out = S;
        if (n_in > 2000000 || n_out > 2000000) continue;
        for (int es : {4, 8}) {
            XposeParams p;
            int vi, vo;
            double eff;
            setup_xpose(rank, ext, si, so, es, &p, &vi, &vo, &eff, in_off, out_off);
            std::vector<int64_t> map(n_out, -1);
            replay(p, vi, vo, n_in, n_out, map, in_off, out_off);
            int64_t hit = 0;
            for (int64_t q = 0; q < n; ++q) {   // view element q (input index order)
                int64_t rem = q, a = in_off, c = out_off;
                for (int d = 0; d < rank; ++d) { const int64_t x = rem % ext[d]; rem /= ext[d]; a += x * si[d]; c += x * so[d]; }
                CHECK(map[c] == a, "view case %d: out %lld from %lld, expected %lld", it, (long long)c,
                      (long long)map[c], (long long)a);
            }
            for (int64_t c = 0; c < n_out; ++c) hit += map[c] >= 0;
            CHECK(hit == n, "view case %d: %lld outputs written, %lld expected", it, (long long)hit, (long long)n);
            ++cases;
        }
    }
    // launch limits on large shapes (extents 8..256, the transpose workload's range): grid below
    // 2^31 blocks, the transposing tile within its 96 KB of shared memory, the element-wise copy
    // stage within the default 48 KB
    for (int it = 0; it < 20000 && fails == 0; ++it) {
        const int rank = it % 2 ? 6 : 4;
        int64_t ext[8], si[8], so[8], so_out[8];
        int perm[8];
        long double tot = 1;
        for (int d = 0; d < rank; ++d) { ext[d] = 8 + rng() % 249; tot *= ext[d]; }
        if (tot > 2147483648.0L) continue;   // the workload's shapes stay at or below 2 GiB
        for (int d = 0; d < rank; ++d) perm[d] = d;
        std::shuffle(perm, perm + rank, rng);
        int64_t s = 1;
        for (int d = 0; d < rank; ++d) { si[d] = s; s *= ext[d]; }
        s = 1;
        for (int d = 0; d < rank; ++d) { so_out[d] = s; s *= ext[perm[d]]; }
        for (int d = 0; d < rank; ++d) so[perm[d]] = so_out[d];
        for (int es : {4, 8}) {
            XposeParams p;
            int vi, vo;
            double eff;
            setup_xpose(rank, ext, si, so, es, &p, &vi, &vo, &eff);
            const uint64_t grid = (uint64_t)p.tiles_u * p.tiles_v * p.tiles_w;
            CHECK(grid < (1ull << 31), "grid of %llu blocks", (unsigned long long)grid);
            if (vo > 0) CHECK(xpose_smem_bytes(p, es) <= 96 * 1024, "tile shared memory %u", xpose_smem_bytes(p, es));
            if ((vo == -1 || (vo == -2 && es == 4)) && !p.single_run)   // rows staged in shared memory
                CHECK((uint64_t)p.tu * p.tw * es <= 48 * 1024, "copy stage of %llu bytes", (unsigned long long)p.tu * p.tw * es);
        }
    }
    // split pre-pass layout: [rows][kpad] with kpad padding (outputs only partly covered)
    for (int it = 0; it < 1500 && fails == 0; ++it) {
        int rank = 2 + rng() % 4;
        int64_t ext[8], si[8], so[8];
        int64_t n = 1;
        for (int d = 0; d < rank; ++d) { ext[d] = 1 + rng() % 40; n *= ext[d]; }
        if (n > 300000) continue;
        int nk = 1 + rng() % (rank - 1);
        std::vector<int> order(rank);
        for (int d = 0; d < rank; ++d) order[d] = d;
        std::shuffle(order.begin(), order.end(), rng);
        int64_t K = 1, R = 1;
        for (int q = 0; q < nk; ++q) K *= ext[order[q]];
        int64_t kpad = (K + 7) / 8 * 8;
        int64_t s = 1;
        for (int d = 0; d < rank; ++d) { si[d] = s; s *= ext[d]; }
        s = 1;
        for (int q = 0; q < nk; ++q) { so[order[q]] = s; s *= ext[order[q]]; }
        s = kpad;
        for (int q = nk; q < rank; ++q) { so[order[q]] = s; s *= ext[order[q]]; R *= ext[order[q]]; }
        XposeParams p;
        int vi, vo;
        double eff;
        setup_xpose(rank, ext, si, so, 4, &p, &vi, &vo, &eff);
        int64_t span = R * kpad;
        std::vector<int64_t> map(span, -1);
        replay(p, vi, vo, n, span, map);
        int64_t written = 0;
        for (int64_t j = 0; j < span; ++j) written += map[j] >= 0;
        CHECK(written == n, "pre-pass wrote %lld of %lld", (long long)written, (long long)n);
        ++cases;
    }
    // GEMM groups of planned contractions: offsets inside their tensors, bijective over M x K
    const char *exprs[] = {"C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", "C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]",
                           "C[a,b,c,d] = A[a,e,b] * B[e,d,c]", "C[i,j] = A[k,i] * B[j,k]",
                           "O[i,j] = x[i] * y[j]", "s[] = x[i] * y[i]"};
    for (const char *e : exprs) {
        for (int prec = 0; prec < 2; ++prec) {
            comet_extent_t ex[8] = {{"i", 3}, {"j", 5}, {"k", 7}, {"a", 6}, {"b", 4}, {"c", 9}, {"d", 2}, {"e", 3}};
            comet_extent_t ex2[2] = {{"f", 5}, {"z", 1}};
            std::vector<comet_extent_t> all(ex, ex + 8);
            all.push_back(ex2[0]);
            comet_dtype_t dt[3] = {COMET_F32, COMET_F32, COMET_F32};
            comet_plan_opts_t o;
            comet_plan_opts_default(&o);
            o.precision = prec ? COMET_PREC_SPLIT_BF16 : COMET_PREC_NATIVE;
            Plan P;
            std::string err;
            if (build_plan(e, all.data(), (int)all.size(), nullptr, 0, dt, 3, &o, &P, &err) != COMET_OK) {
                CHECK(false, "plan failed: %s (%s)", e, err.c_str());
                continue;
            }
            const Step &st = P.steps[0];
            const GemmParams &g = st.gemm;
            int64_t na = P.slots[st.form.swap ? st.b : st.a].elems, nb = P.slots[st.form.swap ? st.a : st.b].elems,
                    nc = P.slots[st.c].elems;
            std::vector<char> seen_a(na, 0), seen_c(nc, 0);
            for (uint32_t m = 0; m < g.M; ++m)
                for (uint32_t k = 0; k < g.K; ++k) {
                    int64_t am, cm, ak, bk;
                    radix_offsets(g.ma, m, am, cm);
                    radix_offsets(g.k, k, ak, bk);
                    CHECK(am + ak >= 0 && am + ak < na, "A offset out of range in %s", e);
                    if (am + ak >= 0 && am + ak < na) seen_a[am + ak]++;
                    CHECK(bk >= 0 && bk < nb, "B K offset out of range");
                }
            for (int64_t q = 0; q < na; ++q) CHECK(seen_a[q] == 1, "A not covered once in %s", e);
            for (uint32_t m = 0; m < g.M; ++m)
                for (uint32_t n2 = 0; n2 < g.N; ++n2) {
                    int64_t am, cm, bn, cn;
                    radix_offsets(g.ma, m, am, cm);
                    radix_offsets(g.nb, n2, bn, cn);
                    CHECK(cm + cn >= 0 && cm + cn < nc, "C offset out of range in %s", e);
                    if (cm + cn >= 0 && cm + cn < nc) seen_c[cm + cn]++;
                }
            for (int64_t q = 0; q < nc; ++q) CHECK(seen_c[q] == 1, "C not covered once in %s", e);
            ++cases;
        }
    }
    // fast division exactness on edge values
    for (uint32_t d : {1u, 2u, 3u, 7u, 24u, 64u, 192u, 12288u, 65535u, 2147483647u, 4294967295u}) {
        FastDiv f = make_fastdiv(d);
        const uint64_t edge[] = {0ull, 1ull, (uint64_t)d - 1, (uint64_t)d, (uint64_t)d + 1, 123456789ull,
                                 4294967295ull, 2147483648ull, 4294967294ull};
        for (uint64_t n : edge) {
            if (n > 4294967295ull) continue;
            CHECK(fd_div((uint32_t)n, f) == (uint32_t)(n / d), "fastdiv %u / %u", (uint32_t)n, d);
        }
        for (int it = 0; it < 20000; ++it) {
            uint32_t n = (uint32_t)rng();
            CHECK(fd_div(n, f) == n / d, "fastdiv %u / %u", n, d);
        }
    }
    std::printf("%d cases, %d failures\n", cases, fails);
    return fails ? 1 : 0;
}
