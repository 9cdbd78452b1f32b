// C ABI (include/comet.h): plan objects, dispatch of plan steps to the kernels, status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/comet.h"
#include "batched.h"
#include "launch.h"
#include "plan.hpp"

struct comet_plan_s {
    comet::Plan p;
};

namespace comet {

__device__ int g_status_word;

static thread_local std::string t_last_error;

static void set_error(const std::string &s) { t_last_error = s; }

int *device_status_word() {
    static std::mutex mu;
    static int *ptrs[128] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<int *>(p);
    }
    return ptrs[dev];
}

// ---- kernel timing ------------------------------------------------------------------------
static const char *kKindNames[] = {"transpose", "scale_copy", "split_prepass", "gemm_split_bf16",
                                   "gemm_f64", "batched_f64", "batched_split", "gemm_emu_bf16x6", "gemv",
                                   "triples_energy", "batched_prepass"};
enum { PK_TRANSPOSE = 0, PK_SCALE, PK_PREPASS, PK_SPLIT, PK_F64, PK_BATCHED_F64, PK_BATCHED_SPLIT, PK_EMU,
       PK_GEMV, PK_TRIPLES, PK_BATCHED_PREPASS, PK_N };

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;

static cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    int idx = -1;
    cudaStream_t s;
    ProfScope(int kind, cudaStream_t st) : s(st) {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        if (!g_prof_on) return;
        ProfRec r{kind, prof_event(), prof_event()};
        if (!r.a || !r.b) return;
        cudaEventRecord(r.a, s);
        g_prof_recs.push_back(r);
        idx = (int)g_prof_recs.size() - 1;
    }
    ~ProfScope() {
        if (idx < 0) return;
        std::lock_guard<std::mutex> lock(g_prof_mu);
        if (idx < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[idx].b, s);
    }
};

// hooks for kernels launched from other files (the batched launch sequence)
int prof_begin(int kind, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (!g_prof_on || kind < 0 || kind >= PK_N) return -1;
    ProfRec r{kind, prof_event(), prof_event()};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    g_prof_recs.push_back(r);
    return (int)g_prof_recs.size() - 1;
}

void prof_end(int idx, cudaStream_t s) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (idx < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[idx].b, s);
}

void set_error_message(const std::string &s) { set_error(s); }

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static comet_status_t cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return COMET_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return COMET_ERR_CUDA;
}

static int64_t timeout_ns(const Plan &P) {
    int64_t ms = P.opts.timeout_ms > 0 ? P.opts.timeout_ms : 2000;
    return ms * 1000000ll;
}

// pointer of a slot at launch time
// pointer of a slot at launch time (inputs and the output: the first element the plan touches)
static void *slot_ptr(const Plan &P, int slot, const void *const *inputs, void *output, void *ws) {
    const Slot &s = P.slots[slot];
    const size_t off = (size_t)s.offset * dtype_size(P.dtype);
    if (s.kind == SLOT_INPUT) return static_cast<char *>(const_cast<void *>(inputs[s.index])) + off;
    if (s.kind == SLOT_OUTPUT) return static_cast<char *>(output) + off;
    return static_cast<char *>(ws) + s.ws_off;
}

// byte range of a slot's buffer at launch time (the stored tensor for inputs and the output,
// the dense intermediate in the workspace): what the debug build's range checks allow
static DbgRange slot_range(const Plan &P, int slot, const void *const *inputs, void *output, void *ws) {
    const Slot &s = P.slots[slot];
    const int64_t es = (int64_t)dtype_size(P.dtype);
    if (s.kind == SLOT_INPUT) return dbg_range(inputs[s.index], s.storage * es);
    if (s.kind == SLOT_OUTPUT) return dbg_range(output, s.storage * es);
    return dbg_range(static_cast<char *>(ws) + s.ws_off, s.elems * es);
}

// max |x| over the elements of a step operand (a strided walk for views)
static cudaError_t operand_absmax(const Slot &s, const void *p, int es, void *out, cudaStream_t stream) {
    if (s.view) return launch_absmax_view(p, s.vradix, es, out, stream);
    return launch_absmax(p, s.elems, es, out, stream);
}

static comet_status_t run_plan(const Plan &P, const void *const *inputs, void *output, void *ws,
                               cudaStream_t stream) {
    int *status = device_status_word();
    if (!status) return cuda_status(cudaErrorNoDevice, "status word");
    const int es = (int)dtype_size(P.dtype);
    for (const Step &st : P.steps) {
        double alpha = 1.0, beta = 0.0;
        if (st.final_step) {
            alpha = P.alpha;
            if (P.op == 1) beta = 1.0;
            if (P.op == 2) { alpha = -alpha; beta = 1.0; }
        }
        void *pa = slot_ptr(P, st.a, inputs, output, ws);
        void *pc = slot_ptr(P, st.c, inputs, output, ws);
        cudaError_t e = cudaSuccess;
        const DbgRange ra = slot_range(P, st.a, inputs, output, ws), rc = slot_range(P, st.c, inputs, output, ws);
        if (st.kernel == KK_COPY) {
            XposeParams x = st.copy;
            x.in = pa; x.out = pc; x.alpha = alpha; x.beta = beta;
            x.dbg_in = ra; x.dbg_out = rc; x.status = status;
            x.plant = (P.opts.debug_flags & 8) ? (int64_t(1) << 40) : 0;
            if (alpha == 1.0 && beta == 0.0) {
                ProfScope ps(PK_TRANSPOSE, stream);
                e = launch_move(x, es, st.copy_vec_in, st.copy_vec_out, stream);
            } else {
                ProfScope ps(PK_SCALE, stream);
                e = launch_scale(x, es, st.copy_vec_in, st.copy_vec_out, stream);
            }
            if (e != cudaSuccess) return cuda_status(e, "copy kernel");
            continue;
        }
        if (st.kernel == KK_REDUCE) {   // sum over labels private to the operand (gemv with v = 1)
            GemvParams v = st.gemv;
            v.X = pa;
            v.v = nullptr;
            v.Y = pc;
            v.dbg_x = ra; v.dbg_v = dbg_range(nullptr, 0); v.dbg_y = rc; v.status = status;
            v.dbg_p = dbg_range(static_cast<char *>(ws) + st.ws_partial, (int64_t)v.n_batch * v.nchunks * v.N * 8);
            v.alpha = alpha;
            v.beta = beta;
            v.partial = reinterpret_cast<double *>(static_cast<char *>(ws) + st.ws_partial);
            {
                ProfScope ps(PK_GEMV, stream);
                e = launch_gemv(v, es, stream);
            }
            if (e != cudaSuccess) return cuda_status(e, "reduction kernel");
            continue;
        }
        void *pb = slot_ptr(P, st.b, inputs, output, ws);
        const DbgRange rb = slot_range(P, st.b, inputs, output, ws);
        char *w = static_cast<char *>(ws);
        void *sc_a = w + st.ws_scales, *sc_b = w + st.ws_scales + 8;
        const bool split_like = st.kernel == KK_GEMM_SPLIT || st.kernel == KK_GEMM_EMU;
        if (split_like) {   // operand scales over the whole operands (every batch index shares them)
            const Slot &sa_ = P.slots[st.form.swap ? st.b : st.a], &sb_ = P.slots[st.form.swap ? st.a : st.b];
            const void *xa = st.form.swap ? pb : pa, *xb = st.form.swap ? pa : pb;
            if (!sa_.view && !sb_.view) {   // both dense: one launch (sc_b is the word after sc_a)
                ProfScope ps(PK_PREPASS, stream);
                e = launch_absmax2(xa, sa_.elems, xb, sb_.elems, es, sc_a, stream);
            } else {
                {
                    ProfScope ps(PK_PREPASS, stream);
                    e = operand_absmax(sa_, xa, es, sc_a, stream);
                }
                if (e == cudaSuccess) {
                    ProfScope ps(PK_PREPASS, stream);
                    e = operand_absmax(sb_, xb, es, sc_b, stream);
                }
            }
            if (e != cudaSuccess) return cuda_status(e, "split pre-pass (scales)");
        }
        // one pass of the step's kernels per batch index (a single pass without batch labels;
        // the gemv kernels take every batch index in one launch)
        const int64_t passes = st.kernel == KK_GEMV ? 1 : st.n_batch;
        for (int64_t bi = 0; bi < passes; ++bi) {
            int64_t oa = 0, ob = 0, oc = 0, r = bi;
            for (size_t d = 0; d < st.bt_ext.size(); ++d) {
                const int64_t x = r % st.bt_ext[d];
                r /= st.bt_ext[d];
                oa += x * st.bt_sa[d];
                ob += x * st.bt_sb[d];
                oc += x * st.bt_sc[d];
            }
            void *qa = static_cast<char *>(pa) + oa * es;
            void *qb = static_cast<char *>(pb) + ob * es;
            void *qc = static_cast<char *>(pc) + oc * es;
            GemmParams g = st.gemm;
            g.A = st.form.swap ? qb : qa;
            g.B = st.form.swap ? qa : qb;
            g.C = qc;
            g.alpha = alpha;
            g.beta = beta;
            g.status = status;
            g.timeout_ns = timeout_ns(P);
            g.dbg_a = st.form.swap ? rb : ra;
            g.dbg_b = st.form.swap ? ra : rb;
            g.dbg_c = rc;
            if (st.kernel == KK_GEMV) {
                GemvParams v = st.gemv;
                v.v = st.gemv_vec_is_a ? g.A : g.B;
                v.X = st.gemv_vec_is_a ? g.B : g.A;
                v.Y = qc;
                v.dbg_v = st.gemv_vec_is_a ? g.dbg_a : g.dbg_b;
                v.dbg_x = st.gemv_vec_is_a ? g.dbg_b : g.dbg_a;
                v.dbg_y = rc;
                v.status = status;
                v.dbg_p = dbg_range(w + st.ws_partial, (int64_t)v.n_batch * v.nchunks * v.N * 8);
                v.alpha = alpha;
                v.beta = beta;
                v.partial = reinterpret_cast<double *>(w + st.ws_partial);
                {
                    ProfScope ps(PK_GEMV, stream);
                    e = launch_gemv(v, es, stream);
                }
                if (e != cudaSuccess) return cuda_status(e, "gemv kernel");
                continue;
            }
            if (st.kernel == KK_GEMM_F64) {
                bool ak = g.k.n > 0 && (g.k.s0[0] == 1 || g.ma.n == 0 || (g.ma.s0[0] != 1 && g.k.s0[0] < g.ma.s0[0]));
                bool bk = g.k.n > 0 && (g.k.s1[0] == 1 || g.nb.n == 0 || (g.nb.s0[0] != 1 && g.k.s1[0] < g.nb.s0[0]));
                {
                    ProfScope ps(PK_F64, stream);
                    e = launch_gemm_f64(g, es, ak, bk, stream);
                }
                if (e != cudaSuccess) return cuda_status(e, "gemm_f64 kernel");
                continue;
            }
            XposeParams xa = st.pre_a, xb = st.pre_b;
            xa.in = g.A; xa.out = w + st.ws_parts_a; xa.scale_bits = sc_a;
            xb.in = g.B; xb.out = w + st.ws_parts_b; xb.scale_bits = sc_b;
            const int64_t n_planes = st.kernel == KK_GEMM_EMU ? 6 : 3;
            xa.dbg_in = g.dbg_a; xa.dbg_out = dbg_range(xa.out, n_planes * xa.out_plane * 2);
            xb.dbg_in = g.dbg_b; xb.dbg_out = dbg_range(xb.out, n_planes * xb.out_plane * 2);
            xa.status = xb.status = status;
            xa.plant = xb.plant = 0;
            auto split = st.kernel == KK_GEMM_EMU ? launch_split6 : launch_split;
            {
                ProfScope ps(PK_PREPASS, stream);
                e = split(xa, es, st.pre_a_vec, st.pre_a_vout, stream);
            }
            if (e != cudaSuccess) return cuda_status(e, "split pre-pass (A)");
            {
                ProfScope ps(PK_PREPASS, stream);
                e = split(xb, es, st.pre_b_vec, st.pre_b_vout, stream);
            }
            if (e != cudaSuccess) return cuda_status(e, "split pre-pass (B)");
            if (st.kernel == KK_GEMM_EMU) {
                ProfScope ps(PK_EMU, stream);
                e = launch_gemm_emu(g, w + st.ws_parts_a, w + st.ws_parts_b, st.kpad, sc_a, sc_b,
                                    P.opts.debug_flags, stream, 0);
                if (e != cudaSuccess) return cuda_status(e, "emulated FP64 gemm kernel");
            } else {
                ProfScope ps(PK_SPLIT, stream);
                e = launch_gemm_split(g, w + st.ws_parts_a, w + st.ws_parts_b, st.kpad, sc_a, sc_b,
                                      P.opts.kc, es, P.opts.debug_flags, stream, 0, st.ksplit,
                                      reinterpret_cast<float *>(w + st.ws_ksplit), (int64_t)st.ksplit_bytes);
                if (e != cudaSuccess) return cuda_status(e, "split gemm kernel");
            }
        }
    }
    return COMET_OK;
}

static bool pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// One slice of a column-major tensor along one label: `height` runs of `width` bytes, `pitch`
// bytes apart, between a strided and a compact or strided layout.  One plain copy when there is
// a single run; a 2-D copy while the pitch is below 2^31; otherwise one copy per run.
static cudaError_t copy_slice(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width,
                              size_t height, cudaMemcpyKind kind, cudaStream_t s) {
    if (height == 1) return cudaMemcpyAsync(dst, src, width, kind, s);
    if (dpitch < (1ull << 31) && spitch < (1ull << 31))
        return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, s);
    for (size_t r = 0; r < height; ++r) {
        cudaError_t e = cudaMemcpyAsync(static_cast<char *>(dst) + r * dpitch,
                                        static_cast<const char *>(src) + r * spitch, width, kind, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// comet_contract_host through the slice pipeline of a one-step split / emulated-FP64 plan (see
// HostPipe): the slices of X and W cross into compact device slices in the planned copy order;
// each slice gets its own scale word and planes, pre-passed before its first GEMM block; block
// (i, j) multiplies W slice i by X slice j (the step's GEMM with both row groups shortened,
// writing the result through the full result strides from the block's first element) in the
// planned block order; results go back on a third stream, block by block when the layout
// allows, else each result slice after its column's last block.  n_calls contractions of the
// same plan run back to back through the same device buffers: the copies of call t + 1 start
// while call t still computes, each slice's copy waiting only for the pre-pass of call t that
// read the slice's device buffer, and each GEMM block waiting only for the copy-out of call t
// that read its result region.
static comet_status_t run_host_pipe(const Plan &P, int n_calls, const void *const *host_in,
                                    void *const *host_out, void *const *dev_in, void *dev_out, void *ws,
                                    cudaStream_t s) {
    const HostPipe &h = P.pipe;
    const Step &st = P.steps[0];
    const size_t es = dtype_size(P.dtype);
    int *status = device_status_word();
    if (!status) return cuda_status(cudaErrorNoDevice, "status word");
    struct Res {
        cudaStream_t cin = nullptr, cout = nullptr;
        std::vector<cudaEvent_t> ev;
        ~Res() {   // the copy streams finish before the call returns (its host buffers stay in use)
            if (cin) cudaStreamSynchronize(cin);
            if (cout) cudaStreamSynchronize(cout);
            for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
            if (cin) cudaStreamDestroy(cin);
            if (cout) cudaStreamDestroy(cout);
        }
    } r;
    const int n = h.n_chunks, nw = h.w_n;
    if (n + nw > 32) return COMET_ERR_INTERNAL;   // one scale word per slice in the 256-byte region
    cudaError_t e = cudaStreamCreateWithFlags(&r.cin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r.cout, cudaStreamNonBlocking);
    // per call: start, end, X copies, column results, W copies, blocks; across calls: the
    // pre-pass of each X and W slice, the copy-out of each block (or column)
    const size_t n_ev = 2 + 2 * n + nw + (size_t)n * nw;
    r.ev.assign(2 * n_ev + n + nw, nullptr);
    for (auto &x : r.ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e, "host pipeline streams");
    cudaEvent_t e0 = r.ev[0], e_end = r.ev[1];
    cudaEvent_t *e_in = &r.ev[2], *e_g = &r.ev[2 + n], *e_w = &r.ev[2 + 2 * n], *e_blk = &r.ev[2 + 2 * n + nw];
    // copy-out done (per block, per column in column mode, and the whole call's): a later call
    // writes a result region only after these
    cudaEvent_t *o_blk = &r.ev[n_ev + 2 + 2 * n + nw], *o_col = &r.ev[n_ev + 2 + n], o_end = r.ev[n_ev + 1];
    cudaEvent_t *p_x = &r.ev[2 * n_ev], *p_w = &r.ev[2 * n_ev + n];   // pre-pass done per slice

    double alpha = P.alpha, beta = 0.0;
    if (P.op == 1) beta = 1.0;
    if (P.op == 2) { alpha = -alpha; beta = 1.0; }
    const bool x_is_b = h.side == 1;
    char *w = static_cast<char *>(ws);
    // scale words: X slices in slots 0, nw + 1, nw + 2, ...; W slices in slots 1 .. nw
    auto sc_x = [&](int j) { return w + st.ws_scales + 8 * (j == 0 ? 0 : nw + j); };
    auto sc_w = [&](int i) { return w + st.ws_scales + 8 * (1 + i); };
    char *parts_x0 = w + (x_is_b ? st.ws_parts_b : st.ws_parts_a);
    char *parts_w0 = w + (x_is_b ? st.ws_parts_a : st.ws_parts_b);
    const bool emu = st.kernel == KK_GEMM_EMU;
    const size_t n_planes = emu ? 6 : 3;
    // every slice's planes sit after those of the slices before it
    auto parts_x = [&](int j) { return parts_x0 + n_planes * (size_t)(h.rows_inner * h.xb[j]) * (size_t)st.kpad * 2; };
    auto parts_w = [&](int i) { return parts_w0 + n_planes * (size_t)(h.w_rows_inner * h.wb[i]) * (size_t)st.kpad * 2; };
    auto split = emu ? launch_split6 : launch_split;
    const char *hx = nullptr, *hw = nullptr;   // the current call's host buffers
    char *hc = nullptr;
    char *dx = static_cast<char *>(dev_in[h.x_in]);
    char *dw = static_cast<char *>(dev_in[h.w_in]);
    char *dc = static_cast<char *>(dev_out);
    const size_t x_unit = (size_t)h.x_inner * h.x_outer * es;      // compact bytes per unit of L
    const size_t w_unit = (size_t)h.w_inner * h.w_outer * es;
    const size_t x_pitch = (size_t)h.x_inner * h.ext * es, c_pitch = (size_t)h.c_inner * h.ext * es;
    const size_t w_pitch = (size_t)h.w_inner * h.w_ext * es;
    auto lx_of = [&](int j) { return h.xb[j + 1] - h.xb[j]; };
    auto lw_of = [&](int i) { return h.wb[i + 1] - h.wb[i]; };
    // a result block is a 3-D box when the result's W label sits directly below or above L
    const bool w_below = h.wc_inner * h.w_ext == h.c_inner;
    auto copy_block = [&](int j, int i) {   // result block (W slice i, X slice j), device to host
        const int64_t l0 = h.xb[j], lc = lx_of(j), m0 = h.wb[i], mc = lw_of(i);
        cudaMemcpy3DParms m = {};
        m.kind = cudaMemcpyDeviceToHost;
        if (w_below) {   // runs over the W label's slice, rows over L, slabs above L
            const size_t pitch = (size_t)h.c_inner * es;
            m.srcPtr = make_cudaPitchedPtr(dc, pitch, pitch, (size_t)h.ext);
            m.dstPtr = make_cudaPitchedPtr(hc, pitch, pitch, (size_t)h.ext);
            m.srcPos = m.dstPos = make_cudaPos((size_t)m0 * h.wc_inner * es, (size_t)l0, 0);
            m.extent = make_cudaExtent((size_t)mc * h.wc_inner * es, (size_t)lc, (size_t)h.c_outer);
        } else {         // runs over L's slice, rows over the W label, slabs above it
            const size_t pitch = (size_t)h.wc_inner * es;
            m.srcPtr = make_cudaPitchedPtr(dc, pitch, pitch, (size_t)h.w_ext);
            m.dstPtr = make_cudaPitchedPtr(hc, pitch, pitch, (size_t)h.w_ext);
            m.srcPos = m.dstPos = make_cudaPos((size_t)l0 * h.c_inner * es, (size_t)m0, 0);
            m.extent = make_cudaExtent((size_t)lc * h.c_inner * es, (size_t)mc, (size_t)(h.c_outer / h.w_ext));
        }
        return cudaMemcpy3DAsync(&m, r.cout);
    };

    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r.cin, e0, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r.cout, e0, 0);
    if (e != cudaSuccess) return cuda_status(e, "host pipeline fork");
    // a later call's copy into a slice's device buffer waits for the pre-pass that read it (the
    // wait is enqueued before this call's pre-pass records the event again)
    auto copy_w = [&](int i, bool later) {
        const int64_t l0 = h.wb[i], lc = lw_of(i);
        const size_t ww = (size_t)h.w_inner * lc * es;
        cudaError_t ee = later ? cudaStreamWaitEvent(r.cin, p_w[i], 0) : cudaSuccess;
        if (ee == cudaSuccess)
            ee = copy_slice(dw + l0 * w_unit, ww, hw + (size_t)l0 * h.w_inner * es, w_pitch, ww,
                            (size_t)h.w_outer, cudaMemcpyHostToDevice, r.cin);
        if (ee == cudaSuccess) ee = cudaEventRecord(e_w[i], r.cin);
        return ee;
    };
    auto copy_x = [&](int j, bool later) {
        const int64_t l0 = h.xb[j], lc = lx_of(j);
        const size_t xw = (size_t)h.x_inner * lc * es;
        cudaError_t ee = later ? cudaStreamWaitEvent(r.cin, p_x[j], 0) : cudaSuccess;
        if (ee == cudaSuccess)
            ee = copy_slice(dx + l0 * x_unit, xw, hx + (size_t)l0 * h.x_inner * es, x_pitch, xw,
                            (size_t)h.x_outer, cudaMemcpyHostToDevice, r.cin);
        if (ee == cudaSuccess && P.op != 0) {   // "+=" / "-=": the result slice in as well, once
            const size_t off = (size_t)l0 * h.c_inner * es;   // the earlier call's copy-out is done
            if (later) ee = cudaStreamWaitEvent(r.cin, o_end, 0);
            if (ee == cudaSuccess)
                ee = copy_slice(dc + off, c_pitch, hc + off, c_pitch, (size_t)h.c_inner * lc * es,
                                (size_t)h.c_outer, cudaMemcpyHostToDevice, r.cin);
        }
        if (ee == cudaSuccess) ee = cudaEventRecord(e_in[j], r.cin);
        return ee;
    };

    // scale and pre-pass of one slice, on the compute stream after its copy
    auto prep = [&](cudaEvent_t ready, char *src, int64_t n_elems, void *scale, const XposeParams &tmpl,
                    int vec, int vout, char *planes, cudaEvent_t done) {
        cudaError_t ee = cudaStreamWaitEvent(s, ready, 0);
        if (ee == cudaSuccess) {
            ProfScope ps(PK_PREPASS, s);
            ee = launch_absmax(src, n_elems, (int)es, scale, s);
        }
        if (ee == cudaSuccess) {
            XposeParams xp = tmpl;
            xp.in = src; xp.out = planes; xp.scale_bits = scale;
            xp.dbg_in = dbg_range(src, n_elems * (int64_t)es);
            xp.dbg_out = dbg_range(planes, (int64_t)n_planes * xp.out_plane * 2);
            xp.status = status;
            xp.plant = 0;
            ProfScope ps(PK_PREPASS, s);
            ee = split(xp, (int)es, vec, vout, s);
        }
        if (ee == cudaSuccess) ee = cudaEventRecord(done, s);
        return ee;
    };
    for (int t = 0; t < n_calls; ++t) {
        const bool later = t > 0;
        hx = static_cast<const char *>(host_in[(size_t)t * P.n_in + h.x_in]);
        hw = static_cast<const char *>(host_in[(size_t)t * P.n_in + h.w_in]);
        hc = static_cast<char *>(host_out[t]);
        // copies in, in the planned order (and the result slices for "+=" / "-=" with X's)
        for (int q : h.copies) {
            e = q >= 0 ? copy_x(q, later) : copy_w(-1 - q, later);
            if (e != cudaSuccess) return cuda_status(e, "host pipeline copy in");
        }
        std::vector<char> done_x(n, 0), done_w(nw, 0);
        std::vector<int> left(n, nw);
        for (int u : h.blocks) {
            const int i = u / n, j = u % n;
            const int64_t l0 = h.xb[j], lc = lx_of(j), m0 = h.wb[i], mc = lw_of(i);
            char *xs = dx + l0 * x_unit, *wsl = dw + m0 * w_unit;
            if (!done_w[i]) {
                e = prep(e_w[i], wsl, h.w_inner * mc * h.w_outer, sc_w(i), h.w_pre[i], h.w_pre_vec[i],
                         h.w_pre_vout[i], parts_w(i), p_w[i]);
                if (e != cudaSuccess) return cuda_status(e, "host pipeline pre-pass (W slice)");
                done_w[i] = 1;
            }
            if (!done_x[j]) {
                e = prep(e_in[j], xs, h.x_inner * lc * h.x_outer, sc_x(j), h.pre[j], h.pre_vec[j], h.pre_vout[j],
                         parts_x(j), p_x[j]);
                if (e != cudaSuccess) return cuda_status(e, "host pipeline pre-pass (X slice)");
                done_x[j] = 1;
            }
            // the earlier call's copy-out of this block's result region is done
            if (later) {
                e = cudaStreamWaitEvent(s, h.blockwise ? o_blk[u] : o_col[j], 0);
                if (e != cudaSuccess) return cuda_status(e, "host pipeline wait");
            }
            GemmParams g = st.gemm;
            Radix &rx = x_is_b ? g.nb : g.ma;
            Radix &rw = x_is_b ? g.ma : g.nb;
            const uint32_t rows_x = (uint32_t)(h.rows_inner * lc), rows_w = (uint32_t)(h.w_rows_inner * mc);
            rx.ext[rx.n - 1] = (uint32_t)lc;
            rx.fd[rx.n - 1] = make_fastdiv((uint32_t)lc);
            rx.total = rows_x;
            rw.ext[rw.n - 1] = (uint32_t)mc;
            rw.fd[rw.n - 1] = make_fastdiv((uint32_t)mc);
            rw.total = rows_w;
            if (x_is_b) { g.N = rows_x; g.M = rows_w; } else { g.M = rows_x; g.N = rows_w; }
            g.A = x_is_b ? static_cast<void *>(wsl) : static_cast<void *>(xs);
            g.B = x_is_b ? static_cast<void *>(xs) : static_cast<void *>(wsl);
            g.C = dc + ((size_t)l0 * h.c_inner + (size_t)m0 * h.wc_inner) * es;
            g.alpha = alpha;
            g.beta = beta;
            g.status = status;
            g.timeout_ns = timeout_ns(P);
            g.dbg_a = g.dbg_b = dbg_range(nullptr, 0);   // read through tensor maps only
            g.dbg_c = dbg_range(dc, (int64_t)P.slots[st.c].storage * (int64_t)es);
            void *pa = x_is_b ? static_cast<void *>(parts_w(i)) : static_cast<void *>(parts_x(j));
            void *pb = x_is_b ? static_cast<void *>(parts_x(j)) : static_cast<void *>(parts_w(i));
            void *sa = x_is_b ? static_cast<void *>(sc_w(i)) : static_cast<void *>(sc_x(j));
            void *sb = x_is_b ? static_cast<void *>(sc_x(j)) : static_cast<void *>(sc_w(i));
            if (emu) {
                ProfScope ps(PK_EMU, s);
                e = launch_gemm_emu(g, pa, pb, st.kpad, sa, sb, P.opts.debug_flags, s, 0);
            } else {
                ProfScope ps(PK_SPLIT, s);
                e = launch_gemm_split(g, pa, pb, st.kpad, sa, sb, P.opts.kc, (int)es, P.opts.debug_flags, s, 0,
                                      st.ksplit, reinterpret_cast<float *>(w + st.ws_ksplit), (int64_t)st.ksplit_bytes);
            }
            if (e != cudaSuccess) return cuda_status(e, "host pipeline gemm");
            if (h.blockwise) {   // this block's result back as soon as it is done
                e = cudaEventRecord(e_blk[u], s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(r.cout, e_blk[u], 0);
                if (e == cudaSuccess) e = copy_block(j, i);
                if (e == cudaSuccess) e = cudaEventRecord(o_blk[u], r.cout);
                if (e != cudaSuccess) return cuda_status(e, "host pipeline copy out (block)");
            } else if (--left[j] == 0) {   // the column's last block: its result slice back
                e = cudaEventRecord(e_g[j], s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(r.cout, e_g[j], 0);
                if (e == cudaSuccess) {
                    const size_t off = (size_t)l0 * h.c_inner * es;
                    e = copy_slice(hc + off, c_pitch, dc + off, c_pitch, (size_t)h.c_inner * lc * es,
                                   (size_t)h.c_outer, cudaMemcpyDeviceToHost, r.cout);
                }
                if (e == cudaSuccess) e = cudaEventRecord(o_col[j], r.cout);
                if (e != cudaSuccess) return cuda_status(e, "host pipeline copy out");
            }
        }
        e = cudaEventRecord(o_end, r.cout);
        if (e != cudaSuccess) return cuda_status(e, "host pipeline copy out");
    }
    e = cudaEventRecord(e_end, r.cout);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e_end, 0);
    if (e != cudaSuccess) return cuda_status(e, "host pipeline join");
    return COMET_OK;
}

}  // namespace comet

using namespace comet;

extern "C" {

comet_status_t comet_plan(const char *expr, const comet_extent_t *extents, int n_extents,
                          const comet_dtype_t *dtypes, int n_dtypes, const comet_plan_opts_t *opts,
                          comet_plan_t *out_plan) {
    if (!out_plan) return COMET_ERR_NULL;
    *out_plan = nullptr;
    comet_plan_s *h = new (std::nothrow) comet_plan_s;
    if (!h) return COMET_ERR_INTERNAL;
    std::string err;
    comet_status_t st;
    try {
        st = build_plan(expr, extents, n_extents, nullptr, 0, dtypes, n_dtypes, opts, &h->p, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
        err = "exception while planning";
    }
    if (st != COMET_OK) {
        set_error(err);
        delete h;
        return st;
    }
    *out_plan = h;
    return COMET_OK;
}

comet_status_t comet_plan_views(const char *expr, const comet_extent_t *extents, int n_extents,
                                const comet_view_t *views, int n_views, const comet_dtype_t *dtypes,
                                int n_dtypes, const comet_plan_opts_t *opts, comet_plan_t *out_plan) {
    if (!out_plan) return COMET_ERR_NULL;
    *out_plan = nullptr;
    comet_plan_s *h = new (std::nothrow) comet_plan_s;
    if (!h) return COMET_ERR_INTERNAL;
    std::string err;
    comet_status_t st;
    try {
        st = build_plan(expr, extents, n_extents, views, n_views, dtypes, n_dtypes, opts, &h->p, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
        err = "exception while planning";
    }
    if (st != COMET_OK) {
        set_error(err);
        delete h;
        return st;
    }
    *out_plan = h;
    return COMET_OK;
}

comet_status_t comet_plan_workspace(comet_plan_t plan, size_t *bytes) {
    if (!plan || !bytes) return COMET_ERR_NULL;
    *bytes = plan->p.batched ? plan->p.batched_ws : plan->p.workspace;
    return COMET_OK;
}

comet_status_t comet_plan_flops(comet_plan_t plan, double *flops) {
    if (!plan || !flops) return COMET_ERR_NULL;
    *flops = plan->p.flops;
    return COMET_OK;
}

comet_status_t comet_plan_flops_natural(comet_plan_t plan, double *flops) {
    if (!plan || !flops) return COMET_ERR_NULL;
    *flops = plan->p.flops_natural;
    return COMET_OK;
}

comet_status_t comet_plan_describe(comet_plan_t plan, char *buf, size_t len) {
    if (!plan || !buf) return COMET_ERR_NULL;
    std::string s = plan->p.batched ? describe_batched(plan->p)
                    : plan->p.triples ? describe_triples(plan->p) : describe_plan(plan->p);
    if (s.size() + 1 > len) return COMET_ERR_ARG;
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return COMET_OK;
}

comet_status_t comet_contract(comet_plan_t plan, const void *const *inputs, void *output, void *workspace,
                              void *stream) {
    if (!plan || !inputs || !output) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (P.batched) { set_error("batched plan: use comet_contract_batched"); return COMET_ERR_ARG; }
    if (P.triples) { set_error("triples plan: use comet_triples_energy"); return COMET_ERR_ARG; }
    for (int i = 0; i < P.n_in; ++i) {
        if (!inputs[i]) return COMET_ERR_NULL;
        if (!aligned16(inputs[i])) return COMET_ERR_ALIGN;
    }
    if (!aligned16(output)) return COMET_ERR_ALIGN;
    if (P.workspace > 0) {
        if (!workspace) return COMET_ERR_WORKSPACE;
        if (!aligned16(workspace)) return COMET_ERR_ALIGN;
    }
    return run_plan(P, inputs, output, workspace, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---- scratch-free contraction --------------------------------------------------------------
// The scratch array behind comet_contract_noalloc().  Host code must not use the name as an
// address (on the host it is only a stand-in for the device symbol); the device address is
// looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[COMET_NOALLOC_MAX_BYTES];

namespace comet {
static void *noalloc_scratch_ptr(comet_status_t *st) {
    static std::mutex mu;
    static void *ptrs[128] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        *st = cuda_status(cudaErrorNoDevice, "no-alloc scratch");
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *st = cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "no-alloc scratch address");
            return nullptr;
        }
        ptrs[dev] = p;
    }
    *st = COMET_OK;
    return ptrs[dev];
}
}  // namespace comet

extern "C" {

comet_status_t comet_contract_noalloc(comet_plan_t plan, const void *const *inputs, void *output,
                                      void *stream) {
    if (!plan || !inputs || !output) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (P.batched) { set_error("batched plan: use comet_contract_batched"); return COMET_ERR_ARG; }
    if (P.triples) { set_error("triples plan: use comet_triples_energy"); return COMET_ERR_ARG; }
    if (P.workspace > COMET_NOALLOC_MAX_BYTES) {
        set_error("plan needs " + std::to_string(P.workspace) + " bytes of scratch; the no-alloc limit is " +
                  std::to_string((size_t)COMET_NOALLOC_MAX_BYTES));
        return COMET_ERR_WORKSPACE;
    }
    for (int i = 0; i < P.n_in; ++i) {
        if (!inputs[i]) return COMET_ERR_NULL;
        if (!aligned16(inputs[i])) return COMET_ERR_ALIGN;
    }
    if (!aligned16(output)) return COMET_ERR_ALIGN;
    comet_status_t st = COMET_OK;
    void *scratch = noalloc_scratch_ptr(&st);
    if (st != COMET_OK) return st;
    return run_plan(P, inputs, output, scratch, static_cast<cudaStream_t>(stream));
}

comet_status_t comet_contract_host_n(comet_plan_t plan, int n_calls, const void *const *host_inputs,
                                     void *const *host_outputs, void *const *dev_inputs, void *dev_output,
                                     void *workspace, void *stream) {
    if (!plan || !host_inputs || !host_outputs || !dev_inputs || !dev_output) return COMET_ERR_NULL;
    if (n_calls < 1) return COMET_ERR_ARG;
    const Plan &P = plan->p;
    if (P.batched || P.triples) return COMET_ERR_ARG;
    for (size_t q = 0; q < (size_t)n_calls * P.n_in; ++q)
        if (!host_inputs[q]) return COMET_ERR_NULL;
    for (int t = 0; t < n_calls; ++t)
        if (!host_outputs[t]) return COMET_ERR_NULL;
    for (int i = 0; i < P.n_in; ++i)
        if (!dev_inputs[i]) return COMET_ERR_NULL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t es = dtype_size(P.dtype);
    if (P.pipe.ok) {   // slice pipeline: pinned host buffers, aligned device buffers
        bool ok = aligned16(dev_output) && (P.workspace == 0 || aligned16(workspace));
        for (int i = 0; i < P.n_in && ok; ++i) ok = aligned16(dev_inputs[i]);
        for (size_t q = 0; q < (size_t)n_calls * P.n_in && ok; ++q) ok = pinned_host(host_inputs[q]);
        for (int t = 0; t < n_calls && ok; ++t) ok = pinned_host(host_outputs[t]);
        if (ok && P.workspace > 0 && !workspace) return COMET_ERR_WORKSPACE;
        if (ok) {
            comet_status_t st = run_host_pipe(P, n_calls, host_inputs, host_outputs, dev_inputs, dev_output,
                                              workspace, s);
            if (st != COMET_OK) return st;
            return comet_sync_status(stream);
        }
    }
    size_t out_bytes = 0;
    bool out_view = false;
    for (auto &sl : P.slots)
        if (sl.kind == SLOT_OUTPUT) { out_bytes = (size_t)sl.storage * es; out_view = sl.view; }
    for (int t = 0; t < n_calls; ++t) {   // every copy and kernel in order on the stream
        for (int i = 0; i < P.n_in; ++i) {
            size_t bytes = (size_t)P.slots[i].storage * es;
            comet_status_t st = cuda_status(cudaMemcpyAsync(dev_inputs[i], host_inputs[(size_t)t * P.n_in + i], bytes,
                                                            cudaMemcpyHostToDevice, s), "input copy");
            if (st != COMET_OK) return st;
        }
        if (P.op != 0 || out_view) {   // read as well, or only partly written (a view)
            comet_status_t st = cuda_status(cudaMemcpyAsync(dev_output, host_outputs[t], out_bytes,
                                                            cudaMemcpyHostToDevice, s), "output copy in");
            if (st != COMET_OK) return st;
        }
        comet_status_t st = comet_contract(plan, const_cast<const void *const *>(dev_inputs), dev_output, workspace,
                                           stream);
        if (st != COMET_OK) return st;
        st = cuda_status(cudaMemcpyAsync(host_outputs[t], dev_output, out_bytes, cudaMemcpyDeviceToHost, s),
                         "output copy");
        if (st != COMET_OK) return st;
    }
    return comet_sync_status(stream);
}

comet_status_t comet_contract_host(comet_plan_t plan, const void *const *host_inputs, void *host_output,
                                   void *const *dev_inputs, void *dev_output, void *workspace, void *stream) {
    if (!host_output) return COMET_ERR_NULL;
    void *outs[1] = {host_output};
    return comet_contract_host_n(plan, 1, host_inputs, outs, dev_inputs, dev_output, workspace, stream);
}

comet_status_t comet_fill(void *out, int64_t n, double value, comet_dtype_t dtype, void *stream) {
    if (n < 0) return COMET_ERR_SHAPE;
    if (n == 0) return COMET_OK;
    if (!out) return COMET_ERR_NULL;
    if (dtype != COMET_F32 && dtype != COMET_F64) return COMET_ERR_DTYPE;
    if (!aligned16(out)) return COMET_ERR_ALIGN;
    return cuda_status(launch_fill(out, n, value, (int)dtype_size(dtype), static_cast<cudaStream_t>(stream)),
                       "fill kernel");
}

comet_status_t comet_transpose(int rank, const int64_t *extents, const int *perm, comet_dtype_t dtype,
                               const void *in, void *out, void *stream) {
    if (!extents || !perm || !in || !out) return COMET_ERR_NULL;
    if (rank < 1 || rank > kMaxRank) return COMET_ERR_ARG;
    if (dtype != COMET_F32 && dtype != COMET_F64) return COMET_ERR_DTYPE;
    int seen[kMaxRank] = {0};
    for (int d = 0; d < rank; ++d) {
        if (perm[d] < 0 || perm[d] >= rank || seen[perm[d]]) return COMET_ERR_ARG;
        seen[perm[d]] = 1;
        if (extents[d] <= 0) return COMET_ERR_SHAPE;
    }
    if (!aligned16(in) || !aligned16(out)) return COMET_ERR_ALIGN;
    int64_t si[kMaxRank], so_out[kMaxRank], so[kMaxRank];
    int64_t s = 1;
    long double tot = 1;
    for (int d = 0; d < rank; ++d) { si[d] = s; s *= extents[d]; tot *= (long double)extents[d]; }
    if (tot > 4.0e12L) return COMET_ERR_SHAPE;
    s = 1;
    for (int d = 0; d < rank; ++d) { so_out[d] = s; s *= extents[perm[d]]; }
    for (int d = 0; d < rank; ++d) so[perm[d]] = so_out[d];
    XposeParams x;
    int vi, vo;
    double eff;
    setup_xpose(rank, extents, si, so, (int)dtype_size(dtype), &x, &vi, &vo, &eff);
    if (x.u.total >= (1u << 31) || x.v.total >= (1u << 31) || x.r.total >= (1u << 31)) return COMET_ERR_SHAPE;
    if ((uint64_t)x.tiles_u * x.tiles_v * x.tiles_w >= (1ull << 31)) {
        set_error("transpose: more than 2^31 tiles");
        return COMET_ERR_SHAPE;
    }
    x.in = in; x.out = out; x.alpha = 1.0; x.beta = 0.0;
    x.dbg_in = dbg_range(in, (int64_t)tot * (int64_t)dtype_size(dtype));
    x.dbg_out = dbg_range(out, (int64_t)tot * (int64_t)dtype_size(dtype));
    x.status = device_status_word();
    x.plant = 0;
    ProfScope ps(PK_TRANSPOSE, static_cast<cudaStream_t>(stream));
    return cuda_status(launch_move(x, (int)dtype_size(dtype), vi, vo, static_cast<cudaStream_t>(stream)),
                       "transpose kernel");
}

comet_status_t comet_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = on != 0;
    return COMET_OK;
}

comet_status_t comet_profile_read(comet_kernel_stat_t *stats, int max_stats, int *n_stats) {
    if (!n_stats || (max_stats > 0 && !stats)) return COMET_ERR_NULL;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    int64_t cnt[PK_N] = {0};
    double tot[PK_N] = {0};
    comet_status_t st = COMET_OK;
    for (auto &r : g_prof_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) st = COMET_ERR_CUDA;
        float ms = 0;
        if (st == COMET_OK && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            cnt[r.kind] += 1;
            tot[r.kind] += ms;
        }
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_recs.clear();
    int n = 0;
    for (int k = 0; k < PK_N; ++k) {
        if (!cnt[k]) continue;
        if (n < max_stats) {
            std::memset(&stats[n], 0, sizeof(stats[n]));
            std::strncpy(stats[n].name, kKindNames[k], sizeof(stats[n].name) - 1);
            stats[n].launches = cnt[k];
            stats[n].total_ms = tot[k];
        }
        ++n;
    }
    *n_stats = n;
    return st;
}

comet_status_t comet_sync_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e, "stream");
    int *w = device_status_word();
    if (!w) return cuda_status(cudaErrorNoDevice, "status word");
    int v = 0, zero = 0;
    e = cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, "status read");
    if (v != 0) {
        e = cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_status(e, "status clear");
        set_error(v == COMET_ERR_BOUNDS ? "a kernel access outside its buffer was skipped (debug build)"
                                        : "a device-side wait ran out of time");
        return static_cast<comet_status_t>(v);
    }
    return COMET_OK;
}

void comet_plan_destroy(comet_plan_t plan) { delete plan; }

const char *comet_status_string(comet_status_t s) {
    switch (s) {
        case COMET_OK: return "ok";
        case COMET_ERR_PARSE: return "parse error";
        case COMET_ERR_LABEL: return "label error";
        case COMET_ERR_SHAPE: return "shape error";
        case COMET_ERR_DTYPE: return "dtype error";
        case COMET_ERR_UNSUPPORTED: return "unsupported";
        case COMET_ERR_ALIGN: return "misaligned pointer";
        case COMET_ERR_NULL: return "null pointer";
        case COMET_ERR_WORKSPACE: return "workspace error";
        case COMET_ERR_CUDA: return "cuda error";
        case COMET_ERR_TIMEOUT: return "device wait timed out";
        case COMET_ERR_INTERNAL: return "internal error";
        case COMET_ERR_ARG: return "bad argument";
        case COMET_ERR_BOUNDS: return "kernel access outside its buffer (debug build)";
    }
    return "unknown status";
}

const char *comet_last_error_message(void) { return t_last_error.c_str(); }

#ifdef COMET_DEBUG
const char *comet_version(void) { return "comet-gb300 0.1 (sm_103a, debug: range-checked kernels)"; }
#else
const char *comet_version(void) { return "comet-gb300 0.1 (sm_103a)"; }
#endif

}  // extern "C"
