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
static bool replay(const XposeParams &p, int vi, int vo, int64_t n_in, int64_t n_out_span,
                   std::vector<int64_t> &src_of_out) {
    const int XT = 256, XTAB = 256;
    const bool copy = vo < 0;
    CHECK(p.tu >= 1 && p.tv >= 1 && p.tw >= 1, "empty tile");
    CHECK((uint64_t)p.tu * p.tv * p.tw <= 8192 + 3 * 256 || (copy && p.tv == 1 && p.tw == 1), "tile too large");
    CHECK((uint64_t)p.tw * p.tv * (p.tu | 1u) * 8 <= 96 * 1024, "tile exceeds the shared memory it is given");
    CHECK(p.tv <= (uint32_t)XTAB && p.tw <= (uint32_t)XTAB, "tile edge above the table size");
    CHECK(copy || p.tu <= (uint32_t)XTAB, "transposing tile edge above the table size");
    const uint64_t grid = (uint64_t)p.tiles_u * p.tiles_v * p.tiles_w;
    const uint32_t tu = p.tu, tv = p.tv, tw = p.tw, pitch = tu | 1u;
    for (uint64_t blk = 0; blk < grid && fails == 0; ++blk) {
        if (copy) {
            const bool affine = tu > (uint32_t)XTAB;
            const uint32_t bu = blk % p.tiles_u, bw = blk / p.tiles_u;
            const uint32_t u0 = bu * tu, w0 = bw * tw;
            const uint32_t nu = std::min(tu, p.u.total - u0), nw = std::min(tw, p.r.total - w0);
            CHECK(!affine || p.u.n == 1, "affine copy of a multi-digit group");
            const int VW = -vo;
            for (uint32_t t = 0; t < (uint32_t)XT; ++t)
                for (uint32_t idx = t * VW; idx < tu * tw; idx += XT * VW) {
                    uint32_t w = fd_div(idx, p.fd_tu), u = idx - w * tu;
                    if (!(u < nu && w < nw)) continue;
                    int64_t a, c, wi, wo;
                    radix_offsets(p.u, u0 + u, a, c);
                    if (affine) { CHECK(a == (int64_t)(u0 + u) * p.u.s0[0] && c == (int64_t)(u0 + u) * p.u.s1[0], "affine offsets"); }
                    radix_offsets(p.r, w0 + w, wi, wo);
                    CHECK((wi + a) % VW == 0 && (wo + c) % VW == 0, "misaligned copy vector");
                    for (int q = 0; q < VW; ++q) {
                        CHECK(u + q < nu, "vector crosses the tile");
                        int64_t a2, c2;
                        radix_offsets(p.u, u0 + u + q, a2, c2);
                        CHECK(a2 == a + q && c2 == c + q, "copy vector not contiguous");
                        int64_t si = wi + a + q, d = wo + c + q;
                        CHECK(si >= 0 && si < n_in && d >= 0 && d < n_out_span, "copy out of bounds");
                        if (d >= 0 && d < n_out_span) { CHECK(src_of_out[d] == -1, "written twice"); src_of_out[d] = si; }
                    }
                }
            continue;
        }
        uint32_t b = blk;
        const uint32_t bu = b % p.tiles_u;
        b /= p.tiles_u;
        const uint32_t bv = b % p.tiles_v, bw = b / p.tiles_v;
        const uint32_t u0 = bu * tu, v0 = bv * tv, w0 = bw * tw;
        const uint32_t nu = std::min(tu, p.u.total - u0), nv = std::min(tv, p.v.total - v0),
                       nw = std::min(tw, p.r.total - w0);
        std::vector<int64_t> ui(tu), uo(tu), vin(tv), vout(tv), wi(tw), wo(tw);
        for (uint32_t i = 0; i < tu; ++i) { ui[i] = uo[i] = 0; if (i < nu) radix_offsets(p.u, u0 + i, ui[i], uo[i]); }
        for (uint32_t i = 0; i < tv; ++i) { vin[i] = vout[i] = 0; if (i < nv) radix_offsets(p.v, v0 + i, vin[i], vout[i]); }
        for (uint32_t i = 0; i < tw; ++i) { wi[i] = wo[i] = 0; if (i < nw) radix_offsets(p.r, w0 + i, wi[i], wo[i]); }
        std::vector<int64_t> buf((size_t)tw * tv * pitch, -1);
        CHECK(p.off32 == 0 || (n_in < (1ll << 31) && n_out_span < (1ll << 31)), "32-bit offsets on a large tensor");
        {   // loads: fixed u per thread, rows (v, w) walked
            const uint32_t lanes = (tu + vi - 1) / vi, rpp = XT / lanes;
            CHECK(rpp >= 1, "no rows per pass (load)");
            for (uint32_t t = 0; t < (uint32_t)XT; ++t) {
                const uint32_t r0 = t / lanes, u = (t - r0 * lanes) * vi;
                if (!(r0 < rpp && u < nu)) continue;
                for (uint32_t row = r0; row < tv * tw; row += rpp) {
                    const uint32_t w = fd_div(row, p.fd_tv), v = row - w * tv;
                    if (!(v < nv && w < nw)) continue;
                    int64_t src = wi[w] + vin[v] + ui[u];
                    CHECK(src % vi == 0, "misaligned vector load");
                    for (int q = 0; q < vi; ++q) {
                        CHECK(u + q < nu, "vector load crosses the tile");
                        CHECK(ui[u + q] == ui[u] + q, "vector load not contiguous");
                        CHECK(src + q >= 0 && src + q < n_in, "load out of bounds");
                        CHECK(row * pitch + u + q < buf.size(), "shared store out of the tile");
                        buf[row * pitch + u + q] = src + q;
                    }
                }
            }
        }
        {   // stores: fixed v per thread, rows (u, w) walked
            const uint32_t lanes = (tv + vo - 1) / vo, rpp = XT / lanes;
            CHECK(rpp >= 1, "no rows per pass (store)");
            for (uint32_t t = 0; t < (uint32_t)XT; ++t) {
                const uint32_t r0 = t / lanes, v = (t - r0 * lanes) * vo;
                if (!(r0 < rpp && v < nv)) continue;
                for (uint32_t row = r0; row < tu * tw; row += rpp) {
                    const uint32_t w = fd_div(row, p.fd_tu), u = row - w * tu;
                    if (!(u < nu && w < nw)) continue;
                    int64_t dst = wo[w] + uo[u] + vout[v];
                    CHECK(dst % vo == 0, "misaligned vector store");
                    for (int q = 0; q < vo; ++q) {
                        CHECK(v + q < nv, "vector store crosses the tile");
                        CHECK(vout[v + q] == vout[v] + q, "vector store not contiguous");
                        size_t bi = (size_t)(w * tv + v + q) * pitch + u;
                        CHECK(bi < buf.size(), "shared load out of the tile");
                        int64_t s2 = buf[bi];
                        CHECK(s2 >= 0, "store of an element that was not loaded");
                        int64_t d = dst + q;
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
        const Fx fx[] = {{1, {5000}, {0}}, {2, {300, 500}, {0, 1}}, {3, {54, 97, 7}, {0, 1, 2}},
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
            if (build_plan(e, all.data(), (int)all.size(), dt, 3, &o, &P, &err) != COMET_OK) {
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
