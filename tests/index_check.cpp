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

// replay of the kernels: returns the output->input map (or empty on failure)
static bool replay(const XposeParams &p, int vi, int vo, int64_t n_in, int64_t n_out_span,
                   std::vector<int64_t> &src_of_out) {
    const int TT = 64, XT = 256;
    bool copy = vo < 0;
    int vw_out = copy ? -vo : vo;
    uint64_t tiles = (uint64_t)p.tiles_u * p.tiles_v;
    uint64_t rch = (p.r.total + p.r_per_cta - 1) / p.r_per_cta;
    uint64_t grid = tiles * rch;
    for (uint64_t b = 0; b < grid; ++b) {
        uint32_t bt = b % tiles, rc = b / tiles;
        uint32_t u0 = (bt % p.tiles_u) * TT, v0 = (bt / p.tiles_u) * TT;
        int64_t u_in[64], u_out[64], v_in[64], v_out[64];
        for (int t = 0; t < TT; ++t) {
            int64_t a = 0, c = 0;
            if (u0 + t < p.u.total) radix_offsets(p.u, u0 + t, a, c);
            u_in[t] = a; u_out[t] = c;
            a = c = 0;
            if (v0 + t < p.v.total) radix_offsets(p.v, v0 + t, a, c);
            v_in[t] = a; v_out[t] = c;
        }
        uint32_t r_begin = rc * p.r_per_cta, r_end = std::min(p.r.total, r_begin + p.r_per_cta);
        for (uint32_t r = r_begin; r < r_end; ++r) {
            int64_t r_in, r_out;
            radix_offsets(p.r, r, r_in, r_out);
            int64_t tile[64][64];
            for (int i = 0; i < 64; ++i) for (int j = 0; j < 64; ++j) tile[i][j] = -1;
            int VI = copy ? vw_out : vi;
            for (int idx = 0; idx < TT * TT / VI; ++idx) {
                int vr = idx / (TT / VI), uc = (idx % (TT / VI)) * VI;
                if (!(v0 + vr < p.v.total && u0 + uc < p.u.total)) continue;
                int64_t src = r_in + v_in[vr] + u_in[uc];
                CHECK(src % VI == 0, "misaligned vector load %lld (w %d)", (long long)src, VI);
                for (int q = 0; q < VI; ++q) {
                    CHECK(u0 + uc + q < p.u.total, "vector load crosses the U extent");
                    int64_t s = src + q;
                    CHECK(s >= 0 && s < n_in, "load out of bounds %lld / %lld", (long long)s, (long long)n_in);
                    CHECK(u_in[uc + q] == u_in[uc] + q, "vector load not contiguous");
                    if (copy) {
                        int64_t d = r_out + v_out[vr] + u_out[uc] + q;
                        CHECK(u_out[uc + q] == u_out[uc] + q, "vector store not contiguous");
                        CHECK(d >= 0 && d < n_out_span, "store out of bounds");
                        if (d >= 0 && d < n_out_span) {
                            CHECK(src_of_out[d] == -1, "output written twice");
                            src_of_out[d] = s;
                        }
                    } else {
                        tile[vr][uc + q] = s;
                    }
                }
            }
            if (copy) continue;
            for (int idx = 0; idx < TT * TT / vo; ++idx) {
                int ur = idx / (TT / vo), vc = (idx % (TT / vo)) * vo;
                if (!(u0 + ur < p.u.total && v0 + vc < p.v.total)) continue;
                int64_t dst = r_out + u_out[ur] + v_out[vc];
                CHECK(dst % vo == 0, "misaligned vector store");
                for (int q = 0; q < vo; ++q) {
                    CHECK(v0 + vc + q < p.v.total, "vector store crosses the V extent");
                    CHECK(v_out[vc + q] == v_out[vc] + q, "vector store not contiguous");
                    int64_t d = dst + q;
                    CHECK(d >= 0 && d < n_out_span, "store out of bounds");
                    CHECK(tile[vc + q][ur] >= 0, "store of a tile element that was not loaded");
                    if (d >= 0 && d < n_out_span) {
                        CHECK(src_of_out[d] == -1, "output written twice");
                        src_of_out[d] = tile[vc + q][ur];
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
