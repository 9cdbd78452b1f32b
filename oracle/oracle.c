/*
 * CPU FP64 oracle for dense tensor contractions — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline arm may load this
 * library.  It shares no code with the GPU path: its own loops, its own index arithmetic,
 * its own generator for the triples weights.
 *
 * What it computes is the plain definition of a tensor contraction in Einstein notation
 * (Section 2 of the COMET paper, the equations for C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]):
 * every output element is the sum, over all values of the labels that appear on the right
 * but not on the left, of the product of the operands.  Multi-operand expressions are summed
 * directly over all non-output labels, so no contraction order is involved (Section 6 states
 * that the order changes the operation count, not the result).
 *
 * Conventions
 *   - Tensors are dense and column-major: the first label of an operand has stride 1.
 *   - Labels are small integers 0 .. n_labels-1; extent[l] is the extent of label l.
 *   - Output element o (column-major linear index over the output labels) gets
 *       out[o] = alpha * sum + beta * out[o]      (beta == 0: out is not read)
 *   - Summation order: the summed labels in order of first appearance on the right-hand
 *     side, the first one fastest; each output is summed sequentially by one thread, so the
 *     result does not depend on the thread count.
 *   - mode 1 ("abs") multiplies absolute values: it gives sum |a||b|..., the scale of the
 *     componentwise error bound.
 *
 * Every entry point returns 0 on success and a negative number on a malformed request.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LABELS 32
#define OR_MAX_OPS 16

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Contraction by the definition: nested loops over the output labels (parallel) and over
 * the summed labels (sequential, odometer order). */
int oracle_einsum(int n_labels, const int64_t *extent,
                  int n_in, const int *rank, const int *labels, const double *const *x,
                  int out_rank, const int *out_labels,
                  double alpha, double beta, int mode,
                  int64_t n_sel, const int64_t *sel, double *out)
{
    if (n_labels <= 0 || n_labels > OR_MAX_LABELS || n_in <= 0 || n_in > OR_MAX_OPS) return -1;
    if (out_rank < 0 || out_rank > OR_MAX_LABELS) return -1;
    for (int l = 0; l < n_labels; ++l) if (extent[l] < 0) return -2;

    /* stride of every label in every operand (a label repeated inside one operand adds its
     * strides: that operand is then read along a diagonal, as the definition says) */
    int64_t *stride = (int64_t *)calloc((size_t)n_in * n_labels, sizeof(int64_t));
    if (!stride) return -3;
    int appears[OR_MAX_LABELS] = {0};
    int first_pos[OR_MAX_LABELS];
    for (int l = 0; l < n_labels; ++l) first_pos[l] = 1 << 30;
    int pos = 0;
    const int *lp = labels;
    for (int t = 0; t < n_in; ++t) {
        int64_t s = 1;
        for (int d = 0; d < rank[t]; ++d) {
            int l = lp[d];
            if (l < 0 || l >= n_labels) { free(stride); return -4; }
            stride[(size_t)t * n_labels + l] += s;
            s *= extent[l];
            appears[l] = 1;
            if (first_pos[l] > pos) first_pos[l] = pos;
            ++pos;
        }
        lp += rank[t];
    }
    int is_out[OR_MAX_LABELS] = {0};
    for (int d = 0; d < out_rank; ++d) {
        int l = out_labels[d];
        if (l < 0 || l >= n_labels || is_out[l] || !appears[l]) { free(stride); return -5; }
        is_out[l] = 1;
    }
    /* summed labels, ordered by first appearance on the right-hand side */
    int sum_lab[OR_MAX_LABELS];
    int n_sum = 0;
    for (int p = 0; p < pos; ++p)
        for (int l = 0; l < n_labels; ++l)
            if (appears[l] && !is_out[l] && first_pos[l] == p) sum_lab[n_sum++] = l;
    int64_t n_out = 1;
    for (int d = 0; d < out_rank; ++d) n_out *= extent[out_labels[d]];
    int64_t n_sum_total = 1;
    for (int q = 0; q < n_sum; ++q) n_sum_total *= extent[sum_lab[q]];
    int64_t n_work = sel ? n_sel : n_out;

    #pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < n_work; ++w) {
        int64_t o = sel ? sel[w] : w;
        int64_t value[OR_MAX_LABELS];
        int64_t base[OR_MAX_OPS];
        /* decode the output index (column-major: first output label fastest) */
        int64_t rem = o;
        for (int d = 0; d < out_rank; ++d) {
            int64_t e = extent[out_labels[d]];
            value[out_labels[d]] = e ? rem % e : 0;
            rem = e ? rem / e : 0;
        }
        for (int t = 0; t < n_in; ++t) {
            int64_t b = 0;
            for (int d = 0; d < out_rank; ++d)
                b += stride[(size_t)t * n_labels + out_labels[d]] * value[out_labels[d]];
            base[t] = b;
        }
        for (int q = 0; q < n_sum; ++q) value[sum_lab[q]] = 0;
        double acc = 0.0;
        for (int64_t s = 0; s < n_sum_total; ++s) {
            double p = 1.0;
            for (int t = 0; t < n_in; ++t) {
                int64_t off = base[t];
                for (int q = 0; q < n_sum; ++q)
                    off += stride[(size_t)t * n_labels + sum_lab[q]] * value[sum_lab[q]];
                double v = x[t][off];
                p *= mode ? fabs(v) : v;
            }
            acc += p;
            /* odometer step over the summed labels, first one fastest */
            for (int q = 0; q < n_sum; ++q) {
                if (++value[sum_lab[q]] < extent[sum_lab[q]]) break;
                value[sum_lab[q]] = 0;
            }
        }
        double r = alpha * acc;
        if (!sel && beta != 0.0) r += beta * out[o];
        out[sel ? w : o] = r;
    }
    free(stride);
    return 0;
}

/* Pure transpose as a bit move (Section 6, "Transpose optimization", computes the same
 * thing): out has extents extent[perm[0]], ..., extent[perm[rank-1]], and the output element
 * with index (j_0, ..., j_{r-1}) is the input element whose index i has i[perm[d]] = j_d.
 * Elements are copied as raw bytes, so NaN payloads, -0.0 and subnormals survive. */
int oracle_transpose(int rank, const int64_t *extent, const int *perm, int elem_bytes,
                     const void *in, void *out, int64_t n_sel, const int64_t *sel)
{
    if (rank <= 0 || rank > OR_MAX_LABELS) return -1;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8) return -2;
    int seen[OR_MAX_LABELS] = {0};
    for (int d = 0; d < rank; ++d) {
        if (perm[d] < 0 || perm[d] >= rank || seen[perm[d]]) return -3;
        seen[perm[d]] = 1;
    }
    int64_t in_stride[OR_MAX_LABELS];
    int64_t s = 1;
    for (int d = 0; d < rank; ++d) { in_stride[d] = s; s *= extent[d]; }
    int64_t n = s;
    int64_t n_work = sel ? n_sel : n;
    const unsigned char *src = (const unsigned char *)in;
    unsigned char *dst = (unsigned char *)out;
    #pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < n_work; ++w) {
        int64_t j = sel ? sel[w] : w;
        int64_t rem = j, off = 0;
        for (int d = 0; d < rank; ++d) {
            int64_t e = extent[perm[d]];
            off += (rem % e) * in_stride[perm[d]];
            rem /= e;
        }
        memcpy(dst + (size_t)(sel ? w : j) * elem_bytes, src + (size_t)off * elem_bytes,
               (size_t)elem_bytes);
    }
    return 0;
}

/* MurmurHash3 32-bit finalizer (Appleby, MurmurHash3, public domain), as published. */
static uint32_t or_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t oracle_fmix32(uint32_t h) { return or_fmix32(h); }

/* One factor of the triples weight: a value in [-1, 1),
 *   h(k, b, x) = (fmix32(k ^ fmix32(b * 0x9E3779B9 + x)) >> 8) * 2^-23 - 1
 * (32-bit unsigned arithmetic with wraparound). */
double oracle_triples_factor(uint32_t key, uint32_t block, uint32_t x) {
    uint32_t h = or_fmix32(key ^ or_fmix32(block * 0x9E3779B9u + x));
    return (double)(h >> 8) * (1.0 / 8388608.0) - 1.0;
}

/* Reduction of one triples block  T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k]  without
 * storing T: s = sum T * W, q = sum T^2.  The weight of element (a,b,c,i,j,k) is the product
 *   W = h(key, block, oA) * h(~key, block, oB)
 * where lin = oA + oB is its column-major linear index in T, oA the part the labels of the
 * first operand (a, b, i) contribute and oB the part of the second operand's labels (c, j, k).
 * ext = {a, b, c, i, j, k, d} extents.  Each element of T is summed over d in order; the
 * partial sums of s and q run over fixed chunks of 4096 elements and the chunk sums are added
 * in order, so the result does not depend on the thread count. */
int oracle_triples_reduce(const int64_t *ext, const double *A, const double *B,
                          uint32_t key, uint32_t block, double *s_out, double *q_out)
{
    int64_t ea = ext[0], eb = ext[1], ec = ext[2], ei = ext[3], ej = ext[4], ek = ext[5],
            ed = ext[6];
    int64_t n = ea * eb * ec * ei * ej * ek;
    const int64_t CH = 4096;
    int64_t n_ch = (n + CH - 1) / CH;
    double *ps = (double *)malloc(sizeof(double) * (size_t)(n_ch ? n_ch : 1));
    double *pq = (double *)malloc(sizeof(double) * (size_t)(n_ch ? n_ch : 1));
    if (!ps || !pq) { free(ps); free(pq); return -3; }
    /* column-major strides of T[a,b,c,i,j,k] */
    const int64_t st_b = ea, st_c = ea * eb, st_i = ea * eb * ec, st_j = st_i * ei, st_k = st_j * ej;
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_ch; ++c) {
        double s = 0.0, q = 0.0;
        int64_t hi = (c + 1) * CH < n ? (c + 1) * CH : n;
        for (int64_t lin = c * CH; lin < hi; ++lin) {
            int64_t r = lin;
            int64_t a = r % ea; r /= ea;
            int64_t b = r % eb; r /= eb;
            int64_t cc = r % ec; r /= ec;
            int64_t i = r % ei; r /= ei;
            int64_t j = r % ej; r /= ej;
            int64_t k = r;
            double t = 0.0;
            for (int64_t d = 0; d < ed; ++d) {
                double av = A[d + ed * (a + ea * (b + eb * i))];      /* A[d,a,b,i] */
                double bv = B[cc + ec * (d + ed * (j + ej * k))];     /* B[c,d,j,k] */
                t += av * bv;
            }
            const int64_t oA = a + st_b * b + st_i * i;
            const int64_t oB = st_c * cc + st_j * j + st_k * k;
            const double w = oracle_triples_factor(key, block, (uint32_t)oA) *
                             oracle_triples_factor(~key, block, (uint32_t)oB);
            s += t * w;
            q += t * t;
        }
        ps[c] = s;
        pq[c] = q;
    }
    double s = 0.0, q = 0.0;
    for (int64_t c = 0; c < n_ch; ++c) { s += ps[c]; q += pq[c]; }
    free(ps);
    free(pq);
    *s_out = s;
    *q_out = q;
    return 0;
}
