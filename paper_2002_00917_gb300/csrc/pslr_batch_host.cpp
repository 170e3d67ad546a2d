// Host side of the batched entry points (include/pslr.h, "batch"): work-item
// assignment and segment streams of the batched apply (pslr_batch.cuh), and
// the batched FGMRES driver over the kernels of pslr_bkrylov.cu, with each
// restart cycle captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "pslr.h"
#include "pslr_internal.h"
#include "pslr_sys.h"
#include "pslr_trace.h"

namespace pslr {
cudaError_t launch_batch_f64(const void *params, int smem, cudaStream_t st);
cudaError_t launch_batch_f32(const void *params, int smem, cudaStream_t st);
cudaError_t launch_batch_f32d(const void *params, int smem, cudaStream_t st);
int coresident_batch_f64(int smem, int nrhs);
int coresident_batch_f32(int smem, int nrhs);
int coresident_batch_f32d(int smem, int nrhs);

// form 0: FP64 in and out; 1: FP32 in and out (BF16 V); 2: FP32 arithmetic on FP64 in and out.
static cudaError_t launch_batch(int form, const void *params, int smem, cudaStream_t st) {
    switch (form) {
    case 0: return launch_batch_f64(params, smem, st);
    case 1: return launch_batch_f32(params, smem, st);
    case 2: return launch_batch_f32d(params, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// Largest cooperative grid of the batched kernel at this shared-memory size
// (the smaller over the forms that share the layout).
static int max_coresident_batch(int smem, bool fp32, int nrhs) {
    if (!fp32) return coresident_batch_f64(smem, nrhs);
    const int a = coresident_batch_f32(smem, nrhs), b = coresident_batch_f32d(smem, nrhs);
    return a < b ? a : b;
}
void bk_spmv_dots(int nchunk, int j, const BkChunk *ch, const BkProb *pr, const BkSys *sys, const double *z,
                  double *w, const double *V, int64_t ld, const BkState &S, cudaStream_t st);
void bk_update(int nchunk, int j, const BkChunk *ch, const BkProb *pr, double *w, const double *V, int64_t ld,
               const double *pin, double *pout, double *hout, int last, const BkState &S, cudaStream_t st);
void bk_hessenberg(int j, int nprob, const BkProb *pr, const BkState &S, cudaStream_t st);
void bk_normalize(int nchunk, const BkChunk *ch, const double *w, double *v, const BkState &S, cudaStream_t st);
void bk_lsq(int nprob, const BkState &S, cudaStream_t st);
void bk_gemv_add(int nchunk, const BkChunk *ch, const double *Z, int64_t ld, double *x, const BkState &S,
                 cudaStream_t st);
void bk_residual(int nchunk, const BkChunk *ch, const BkProb *pr, const BkSys *sys, const double *x,
                 const double *b, double *r, const BkState &S, cudaStream_t st);
void bk_restart(int first, int nprob, const BkProb *pr, const BkState &S, cudaStream_t st);
void bk_start(int nchunk, const BkChunk *ch, const double *r, double *v, const BkState &S, cudaStream_t st);
void launch_axpy(int n, double a, const double *x, double *y, cudaStream_t st);
}  // namespace pslr

using namespace pslr;

namespace {
thread_local std::string g_create_error;  // message of the last failed pslr_batch_create
}

struct pslr_batch {
    int nsys = 0, nrhs = 0, nprob = 0;
    int64_t n_total = 0;
    std::vector<pslr_ctx *> ctx;
    std::vector<SysExport> sx;
    std::vector<int64_t> voff;
    int max_p = 0, max_q = 0, max_m = 0, any_lr = 0, items = 0, grid = 0;
    int group_req[2] = {0, 0};                 // requested items per group, [FP64, FP32] (0: largest that fits)
    int ring_max[2] = {0, 0};                  // cap on the apply's ring slots (0: as many as fit)
    int kchunk = kBkChunk;                     // rows per chunk of the batched Krylov kernels
    int pair64 = 1;                            // FP64 with several rhs: a thread per (row, rhs) pair
    int group[2] = {0, 0}, ngroups[2] = {0, 0};  // items per group and groups, [FP64, FP32]
    int xs[2] = {0, 0}, gs[2] = {0, 0};        // group vector strides
    int ring[2] = {0, 0}, slot_bytes[2] = {0, 0}, smem[2] = {0, 0};
    int64_t apply_bytes[2] = {0, 0};
    // device: merged segments, groups, assignment, streams, per-system parameters and scratch
    char *d_seg[2] = {nullptr, nullptr};
    BatchGroup *d_groups[2] = {nullptr, nullptr};
    int32_t *d_group_off[2] = {nullptr, nullptr};
    int32_t *d_pairs = nullptr, *d_pair_off = nullptr;
    StreamEnt *d_stream[2] = {nullptr, nullptr};
    int64_t *d_stream_off[2] = {nullptr, nullptr};
    void *d_sys[2] = {nullptr, nullptr};  // BatchSys<double>[nsys], BatchSys<float>[nsys]
    void *d_scratch = nullptr;
    unsigned *d_bar = nullptr;
    int *d_err = nullptr;
    long long wait_limit = 1ll << 22;
    // batched FGMRES
    int nchunk = 0;
    BkChunk *d_chunks = nullptr;
    BkProb *d_probs = nullptr;
    BkSys *d_bsys = nullptr;
    int kK = 0;  // restart length the workspace is sized for
    double *d_V = nullptr, *d_Z = nullptr, *d_w = nullptr, *d_r = nullptr, *d_b = nullptr, *d_x = nullptr;
    void *d_state = nullptr;
    BkState S{};
    cudaStream_t cap = nullptr;
    std::map<std::tuple<int, int, long long>, cudaGraphExec_t> graphs;  // (form, restart, wait limit)
    int graph_used = 0;
    std::vector<BkProb> h_probs;       // host copy of the problem table
    std::vector<cudaStream_t> hstream;  // per system: stream of the problems finished on it
    std::vector<double *> he;           // per system: correction of one such problem
    int handoff = 0;                    // problems the last solve finished on their systems
    std::string err;
};

namespace {

pslr_status bfail(pslr_batch *b, pslr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_error = buf;
    return st;
}

#define BCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return bfail(bt, PSLR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class X>
cudaError_t upload(X **dst, const std::vector<X> &src) {
    const size_t bytes = sizeof(X) * std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaMemset(*dst, 0, bytes);
    return cudaMemcpy(*dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice);
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

void free_krylov(pslr_batch *bt) {
    for (auto &kv : bt->graphs) cudaGraphExecDestroy(kv.second);
    bt->graphs.clear();
    dfree(bt->d_V); dfree(bt->d_Z); dfree(bt->d_w); dfree(bt->d_r); dfree(bt->d_b); dfree(bt->d_x);
    dfree(bt->d_state);
    for (double *&e : bt->he) {
        dfree(e);
        e = nullptr;
    }
    bt->d_V = bt->d_Z = bt->d_w = bt->d_r = bt->d_b = bt->d_x = nullptr;
    bt->d_state = nullptr;
    bt->kK = 0;
}

void free_batch(pslr_batch *bt) {
    free_krylov(bt);
    dfree(bt->d_pairs); dfree(bt->d_pair_off);
    for (int p = 0; p < 2; ++p) {
        dfree(bt->d_seg[p]);
        dfree(bt->d_groups[p]);
        dfree(bt->d_group_off[p]);
        dfree(bt->d_stream[p]);
        dfree(bt->d_stream_off[p]);
        dfree(bt->d_sys[p]);
    }
    dfree(bt->d_scratch); dfree(bt->d_bar); dfree(bt->d_err);
    dfree(bt->d_chunks); dfree(bt->d_probs); dfree(bt->d_bsys);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    for (cudaStream_t h : bt->hstream)
        if (h) cudaStreamDestroy(h);
}

// ------------------------------------------------- merged segments of a group

// Host record of one merged segment.
struct SegDesc {
    int64_t off;
    int32_t bytes;
};

// One row of a parsed segment: output row, entries (padding included) and
// the value of the record's last slot (1/diagonal, or 1).
template <class T>
struct PRow {
    int32_t row;
    int32_t zero;  // the zero slot this row's padding entries point at
    std::vector<int32_t> col;
    std::vector<T> val;
    T dinv;
};

// Append the rows of one packed segment (layout of pslr_internal.h) to out,
// with row indices shifted by rs, local column indices by cs (global columns
// are kept), and padding pointed at zero.
template <class T, class IDX>
void parse_segment(const char *seg, int rs, int cs, int zero, std::vector<PRow<T>> &out, bool *diag) {
    SegHdr h;
    std::memcpy(&h, seg, sizeof(h));
    *diag = (h.flags & kSegDiag) != 0;
    const bool global = (h.flags & kSegGlobalCols) != 0;
    const int n = h.n, np = h.np;
    const char *p = seg + sizeof(SegHdr);
    auto col_of = [&](IDX c) { return global ? (int32_t)c : (int32_t)c + cs; };
    if (h.fmt != kTile) {
        const int K = h.fmt;
        const IDX *idx = reinterpret_cast<const IDX *>(p);
        const T *val = reinterpret_cast<const T *>(p + (size_t)np * rec_idx_bytes<IDX>(K));
        for (int j = 0; j < n; ++j) {
            PRow<T> r;
            r.row = (int32_t)idx[(size_t)j * (K + 1)] + rs;
            r.zero = zero;
            for (int k = 0; k < K; ++k) {
                r.col.push_back(col_of(idx[(size_t)j * (K + 1) + 1 + k]));
                r.val.push_back(val[(size_t)j * (K + 1) + k]);
            }
            r.dinv = val[(size_t)j * (K + 1) + K];
            out.push_back(std::move(r));
        }
        return;
    }
    const int w = h.w;
    const T *vals = reinterpret_cast<const T *>(p);
    const T *dinv = reinterpret_cast<const T *>(p + (size_t)np * w * sizeof(T));
    const IDX *cols = reinterpret_cast<const IDX *>(p + (size_t)np * w * sizeof(T) + (*diag ? np * sizeof(T) : 0));
    const uint16_t *rws = reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(cols) +
                                                             (size_t)np * w * sizeof(IDX));
    for (int j = 0; j < n; ++j) {
        PRow<T> r;
        r.row = (int32_t)rws[j] + rs;
        r.zero = zero;
        for (int k = 0; k < w; ++k) {
            r.col.push_back(col_of(cols[(size_t)k * np + j]));
            r.val.push_back(vals[(size_t)k * np + j]);
        }
        r.dinv = *diag ? dinv[j] : T(1);
        out.push_back(std::move(r));
    }
}

// Pack rows [b, e) as one segment (same encodings as the set-up's packer);
// values are copied bit for bit.
template <class T, class IDX>
void pack_prows(std::vector<char> &bytes, std::vector<SegDesc> &desc, const std::vector<PRow<T>> &rows,
                size_t b, size_t e, bool diag, bool global) {
    const int n = (int)(e - b);
    int w = 0;
    for (size_t i = b; i < e; ++i) w = std::max<int>(w, (int)rows[i].col.size());
    const int np = seg_npad(n);
    const int64_t nbytes = seg_bytes<T, IDX>(n, w, diag);
    SegDesc d;
    d.off = (int64_t)bytes.size();
    d.bytes = (int32_t)nbytes;
    bytes.resize(bytes.size() + nbytes, 0);
    char *base = bytes.data() + d.off;
    SegHdr h;
    std::memset(&h, 0, sizeof(h));
    h.n = (uint16_t)n;
    h.flags = (uint8_t)((diag ? (unsigned)kSegDiag : 0u) | (global ? (unsigned)kSegGlobalCols : 0u));
    h.np = (uint16_t)np;
    const int fmt = seg_fmt_for(w);
    h.fmt = (uint8_t)fmt;
    h.w = (uint8_t)(fmt != kTile ? fmt : w);
    h.bytes = (uint32_t)nbytes;
    std::memcpy(base, &h, sizeof(h));
    base += sizeof(SegHdr);
    const int zero0 = rows[b].zero;
    if (fmt != kTile) {
        const int K = fmt;
        IDX *idx = reinterpret_cast<IDX *>(base);
        T *val = reinterpret_cast<T *>(base + (size_t)np * rec_idx_bytes<IDX>(K));
        for (int j = 0; j < np; ++j) {
            const PRow<T> *R = j < n ? &rows[b + j] : nullptr;
            IDX *ir = idx + (size_t)j * (K + 1);
            T *vr = val + (size_t)j * (K + 1);
            ir[0] = R ? (IDX)R->row : (IDX)0;
            for (int k = 0; k < K; ++k) {
                const bool has = R && k < (int)R->col.size();
                ir[1 + k] = has ? (IDX)R->col[k] : (IDX)(R ? R->zero : zero0);
                vr[k] = has ? R->val[k] : T(0);
            }
            vr[K] = R ? R->dinv : T(1);
        }
    } else {
        T *vals = reinterpret_cast<T *>(base);
        T *dinv = reinterpret_cast<T *>(base + (size_t)np * w * sizeof(T));
        IDX *cols = reinterpret_cast<IDX *>(base + (size_t)np * w * sizeof(T) + (diag ? np * sizeof(T) : 0));
        uint16_t *rws = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(cols) + (size_t)np * w * sizeof(IDX));
        for (int j = 0; j < np; ++j) {
            const PRow<T> *R = j < n ? &rows[b + j] : nullptr;
            for (int k = 0; k < w; ++k) {
                const bool has = R && k < (int)R->col.size();
                vals[(size_t)k * np + j] = has ? R->val[k] : T(0);
                cols[(size_t)k * np + j] = has ? (IDX)R->col[k] : (IDX)(R ? R->zero : zero0);
            }
            if (diag) dinv[j] = R ? R->dinv : T(0);
            rws[j] = R ? (uint16_t)R->row : (uint16_t)0;
        }
    }
    desc.push_back(d);
}

// Rows into segments of at most kSegMaxRows rows and kSegBudget bytes.
template <class T, class IDX>
int pack_prow_list(std::vector<char> &bytes, std::vector<SegDesc> &desc, const std::vector<PRow<T>> &rows,
                   bool diag, bool global) {
    int cnt = 0;
    size_t b = 0;
    while (b < rows.size()) {
        size_t e = b;
        int w = 0;
        while (e < rows.size() && (int)(e - b) < kSegMaxRows) {
            const int w2 = std::max<int>(w, (int)rows[e].col.size());
            if (e > b && seg_bytes<T, IDX>((int)(e - b + 1), w2, diag) > kSegBudget) break;
            w = w2;
            ++e;
        }
        pack_prows<T, IDX>(bytes, desc, rows, b, e, diag, global);
        ++cnt;
        b = e;
    }
    return cnt;
}

// Host copies of every system's forward segments of one precision.
pslr_status download_segments(pslr_batch *bt, int prec, std::vector<std::vector<char>> &host) {
    host.resize(bt->nsys);
    for (int k = 0; k < bt->nsys; ++k) {
        host[k].resize((size_t)bt->sx[k].seg_bytes[prec]);
        if (!host[k].empty())
            BCK(cudaMemcpy(host[k].data(), bt->sx[k].seg[prec], host[k].size(), cudaMemcpyDeviceToHost));
    }
    return PSLR_OK;
}

// The merged segments of one group, category by category (kE .. kC2): level
// j of a sweep holds segment j of every item (items are independent, so any
// rows of one merged level may run together); the products take all rows of
// all items.  Returns the merged counts in g.cnt.
template <class T>
void merge_group(const pslr_batch *bt, int prec, const std::vector<char> &host, BatchGroup &g,
                 std::vector<char> &bytes, std::vector<SegDesc> &desc) {
    const SysExport &e = bt->sx[g.sys];
    for (int cat = 0; cat < kNCnt; ++cat) {
        const bool interior_rows = cat == kE || cat == kB1 || cat == kB2;
        const bool global = cat == kCg;
        const bool sweep = cat >= kB1;
        std::vector<std::vector<StreamEnt>> segs(g.n);
        size_t nmax = 0;
        for (int t = 0; t < g.n; ++t) {
            sys_segments(bt->ctx[g.sys], prec, g.sub[t], cat, 0, segs[t]);
            if (sweep) {  // a sweep segment holds consecutive levels: one entry per level block
                std::vector<StreamEnt> blocks;
                for (const StreamEnt &se : segs[t]) {
                    for (int64_t off = se.off; off < se.off + se.bytes;) {
                        SegHdr h;
                        std::memcpy(&h, host.data() + off, sizeof h);
                        StreamEnt b;
                        b.off = off;
                        b.bytes = (int32_t)h.bytes;
                        b.pad = 0;
                        blocks.push_back(b);
                        if (!(h.flags & kSegMore) || h.bytes == 0) break;
                        off += h.bytes;
                    }
                }
                segs[t].swap(blocks);
            }
            nmax = std::max(nmax, segs[t].size());
        }
        int cnt = 0;
        std::vector<PRow<T>> rows;
        bool diag = false;
        auto flush = [&]() {
            if (rows.empty()) return;
            cnt += global ? pack_prow_list<T, int32_t>(bytes, desc, rows, diag, true)
                          : pack_prow_list<T, uint16_t>(bytes, desc, rows, diag, false);
            rows.clear();
        };
        for (size_t j = 0; j < nmax; ++j) {
            for (int t = 0; t < g.n; ++t) {
                if (j >= segs[t].size()) continue;
                const int i = g.sub[t];
                const int p = bt->sx[g.sys].ioff_h[i + 1] - bt->sx[g.sys].ioff_h[i];
                const int q = bt->sx[g.sys].goff_h[i + 1] - bt->sx[g.sys].goff_h[i];
                // rows: interior (E, B) or interface (F, C_g, C0); columns: interior (B, F),
                // interface (E, C0) or global (C_g)
                const int rs = interior_rows ? g.xo[t] : g.go[t];
                const bool col_interior = cat == kF || cat == kB1 || cat == kB2;
                const int cs = col_interior ? g.xo[t] : g.go[t];
                const int zero = global ? e.q : (col_interior ? g.xo[t] + p : g.go[t] + q);
                const char *seg = host.data() + segs[t][j].off;
                if (global) parse_segment<T, int32_t>(seg, rs, cs, zero, rows, &diag);
                else parse_segment<T, uint16_t>(seg, rs, cs, zero, rows, &diag);
            }
            if (sweep) flush();  // one merged level per item segment index
        }
        flush();
        g.cnt[cat] = cnt;
    }
}

// Phase costs of a group in level steps (one merged segment = one step),
// plus a charge for gathers, scatters and low-rank reductions per item.
// Phases: 0, 1 (low rank), the series terms 1..max_m, final.
std::vector<double> group_cost(const pslr_batch *bt, const BatchGroup &g) {
    const SysExport &e = bt->sx[g.sys];
    const int nph = 3 + bt->max_m;
    std::vector<double> c(nph, 0.0);
    const int *n = g.cnt;
    const double nr = bt->nrhs, per = g.n * 2.0;
    c[0] = n[kB1] + n[kB2] + n[kF] + 4 * per + (e.r > 0 ? per * nr * (1 + e.r / 8.0) : n[kC1] + n[kC2]);
    if (e.r > 0) c[1] = n[kC1] + n[kC2] + per * nr * (1 + e.r / 16.0);
    for (int kk = 1; kk <= e.m; ++kk) c[1 + kk] = n[kE] + n[kB1] + n[kB2] + n[kF] + n[kCg] + n[kC1] + n[kC2] + 2 * per;
    c[nph - 1] = n[kE] + n[kB1] + n[kB2] + 4 * per;
    return c;
}

}  // namespace

// ------------------------------------------------------------------ create

// Groups of up to G consecutive subdomains per system, sizes balanced within
// the system; returns the largest group vector lengths through xs, gs.
static std::vector<BatchGroup> form_groups(const pslr_batch *bt, int G, int *xs, int *gs) {
    std::vector<BatchGroup> out;
    *xs = *gs = 1;
    for (int k = 0; k < bt->nsys; ++k) {
        const SysExport &e = bt->sx[k];
        const int ng = (e.s + G - 1) / G;
        for (int a = 0; a < ng; ++a) {
            const int i0 = (int)((int64_t)e.s * a / ng), i1 = (int)((int64_t)e.s * (a + 1) / ng);
            BatchGroup g;
            std::memset(&g, 0, sizeof(g));
            g.sys = k;
            g.n = i1 - i0;
            g.xo[0] = g.go[0] = 0;
            for (int t = 0; t < g.n; ++t) {
                const int i = i0 + t;
                g.sub[t] = i;
                g.xo[t + 1] = g.xo[t] + (e.ioff_h[i + 1] - e.ioff_h[i]) + 1;
                g.go[t + 1] = g.go[t] + (e.goff_h[i + 1] - e.goff_h[i]) + 1;
            }
            *xs = std::max(*xs, g.xo[g.n]);
            *gs = std::max(*gs, g.go[g.n]);
            out.push_back(g);
        }
    }
    return out;
}

static pslr_status batch_build(pslr_batch *bt) {
    const int nsys = bt->nsys, nr = bt->nrhs;
    // sizes and offsets
    bt->voff.resize(nsys);
    int64_t off = 0;
    for (int k = 0; k < nsys; ++k) {
        const SysExport &e = bt->sx[k];
        bt->voff[k] = off;
        off += (int64_t)e.n * nr;
        bt->max_p = std::max(bt->max_p, e.max_p);
        bt->max_q = std::max(bt->max_q, e.max_q);
        bt->max_m = std::max(bt->max_m, e.m);
        bt->any_lr |= e.r > 0;
        bt->items += e.s;
    }
    bt->n_total = off;
    bt->nprob = nsys * nr;
    int dev = 0, optin = 227 * 1024;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

    // groups, merged segments and shared-memory layout per precision
    std::vector<std::vector<BatchGroup>> groups(2);
    std::vector<std::vector<char>> mbytes(2);
    std::vector<std::vector<SegDesc>> mdesc(2);
    std::vector<std::vector<int32_t>> gfirst(2);  // first merged descriptor of each group
    int grid = 1 << 30;
    for (int prec = 0; prec < 2; ++prec) {
        const int ts = prec == 0 ? 8 : 4;
        int item_slot = 128;
        for (int k = 0; k < nsys; ++k) item_slot = std::max(item_slot, bt->sx[k].slot_bytes[prec]);
        // largest group size whose vectors and a 4-slot ring of merged segments fit
        int G = bt->group_req[prec] > 0 ? std::min(bt->group_req[prec], kMaxGroup) : kMaxGroup, xs = 1, gs = 1;
        for (; G >= 1; --G) {
            groups[prec] = form_groups(bt, G, &xs, &gs);
            const int slot_est = std::min(kSegBudget, align_up(G * item_slot, 128));
            const int need = 1024 + smem_fixed(nr * xs - 1, nr * gs - 1, ts, false) + 4 * slot_est;
            if (need <= optin && xs < 65536 && gs < 65536) break;
        }
        if (G < 1)
            return bfail(bt, PSLR_ERR_TOO_LARGE,
                         "batch: %d right-hand sides of the largest subdomain (%d interior, %d interface "
                         "unknowns) do not fit one CTA's shared memory",
                         nr, bt->max_p, bt->max_q);
        bt->group[prec] = G;
        bt->xs[prec] = xs;
        bt->gs[prec] = gs;
        std::vector<std::vector<char>> host;
        pslr_status st = download_segments(bt, prec, host);
        if (st != PSLR_OK) return st;
        for (BatchGroup &g : groups[prec]) {
            gfirst[prec].push_back((int32_t)mdesc[prec].size());
            if (prec == 0) merge_group<double>(bt, prec, host[g.sys], g, mbytes[prec], mdesc[prec]);
            else merge_group<float>(bt, prec, host[g.sys], g, mbytes[prec], mdesc[prec]);
        }
        int sb = 128;
        for (const SegDesc &d : mdesc[prec]) sb = std::max(sb, (int)d.bytes);
        sb = align_up(sb, 128);
        bt->slot_bytes[prec] = sb;
        const int avail = optin - 1024 - smem_fixed(nr * xs - 1, nr * gs - 1, ts, false);
        bt->ring[prec] = std::min(kMaxRing, avail / sb);
        if (bt->ring_max[prec] > 0) bt->ring[prec] = std::min(bt->ring[prec], bt->ring_max[prec]);
        if (bt->ring[prec] < 2)
            return bfail(bt, PSLR_ERR_TOO_LARGE, "batch: no room for the segment ring (%d-byte slots)", sb);
        bt->smem[prec] = smem_layout(sb, bt->ring[prec], nr * xs - 1, nr * gs - 1, ts, false).total;
        const int g = max_coresident_batch(bt->smem[prec], prec == 1, nr);
        if (g < 1) return bfail(bt, PSLR_ERR_CUDA, "batch: the apply kernel cannot be made resident");
        grid = std::min(grid, g);
        bt->ngroups[prec] = (int)groups[prec].size();
    }
    grid = std::min(grid, std::max(bt->ngroups[0], bt->ngroups[1]));
    bt->grid = grid;

    // per precision: groups to CTAs (longest first onto the CTA that raises
    // the sum of the per-phase maxima least: phases are separated by grid
    // barriers, so each phase is balanced, not only the total), then streams
    const int nph = 3 + bt->max_m;
    for (int prec = 0; prec < 2; ++prec) {
        std::vector<BatchGroup> &gl = groups[prec];
        std::vector<int> order(gl.size());
        std::vector<std::vector<double>> cost(gl.size());
        std::vector<double> tot(gl.size(), 0.0);
        for (size_t u = 0; u < gl.size(); ++u) {
            order[u] = (int)u;
            cost[u] = group_cost(bt, gl[u]);
            for (double v : cost[u]) tot[u] += v;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tot[a] > tot[b]; });
        std::vector<std::vector<double>> load(grid, std::vector<double>(nph, 0.0));
        std::vector<double> ctot(grid, 0.0), mx(nph, 0.0);
        std::vector<std::vector<int>> own(grid);
        for (int u : order) {
            int best = 0;
            double bd = 1e300, bl = 1e300;
            for (int b = 0; b < grid; ++b) {
                double d = 0.0;
                for (int ph = 0; ph < nph; ++ph) d += std::max(0.0, load[b][ph] + cost[u][ph] - mx[ph]);
                if (d < bd || (d == bd && ctot[b] < bl)) {
                    bd = d;
                    bl = ctot[b];
                    best = b;
                }
            }
            for (int ph = 0; ph < nph; ++ph) {
                load[best][ph] += cost[u][ph];
                mx[ph] = std::max(mx[ph], load[best][ph]);
            }
            ctot[best] += tot[u];
            own[best].push_back(u);
        }
        std::vector<BatchGroup> hg;
        std::vector<int32_t> hoff(grid + 1, 0);
        std::vector<StreamEnt> ent;
        std::vector<int64_t> soff(grid + 1, 0);
        auto add = [&](int u, std::initializer_list<int> cats) {
            const BatchGroup &g = gl[u];
            for (int cat : cats) {
                int d = gfirst[prec][u];
                for (int k = 0; k < cat; ++k) d += g.cnt[k];
                for (int t = 0; t < g.cnt[cat]; ++t) {
                    StreamEnt e;
                    e.off = mdesc[prec][d + t].off;
                    e.bytes = mdesc[prec][d + t].bytes;
                    e.pad = g.sys;  // the producer skips by system
                    ent.push_back(e);
                }
            }
        };
        for (int b = 0; b < grid; ++b) {
            hoff[b] = (int32_t)hg.size();
            for (int u : own[b]) hg.push_back(gl[u]);
            soff[b] = (int64_t)ent.size();
            for (int u : own[b]) {
                add(u, {kB1, kB2, kF});
                if (bt->sx[gl[u].sys].r == 0) add(u, {kC1, kC2});
            }
            if (bt->any_lr)
                for (int u : own[b])
                    if (bt->sx[gl[u].sys].r > 0) add(u, {kC1, kC2});
            for (int kk = 1; kk <= bt->max_m; ++kk)
                for (int u : own[b])
                    if (bt->sx[gl[u].sys].m >= kk) add(u, {kE, kB1, kB2, kF, kCg, kC1, kC2});
            for (int u : own[b]) add(u, {kE, kB1, kB2});
        }
        hoff[grid] = (int32_t)hg.size();
        soff[grid] = (int64_t)ent.size();
        int64_t seg_bytes = 0;
        for (const StreamEnt &e : ent) seg_bytes += e.bytes;
        // algorithmic bytes: every segment of the stream once, V once per pass,
        // and per right-hand side the vectors of the single-system count
        const int64_t vs = prec == 0 ? 8 : 4, vb = prec == 0 ? 8 : 2;
        int64_t bytes = seg_bytes;
        for (int k = 0; k < nsys; ++k) {
            const SysExport &e = bt->sx[k];
            const int64_t m = e.m, r = e.r, q = e.q;
            bytes += 2 * q * r * vb;
            int64_t vec = 2 * (int64_t)e.p + q + e.n;
            vec += (r > 0 ? 2 * q : 0) + 2 * q;
            vec += m * (q + q + 2 * q);
            bytes += vec * vs * nr;
        }
        bt->apply_bytes[prec] = bytes;
        if (mbytes[prec].empty()) mbytes[prec].resize(16, 0);
        BCK(upload(&bt->d_seg[prec], mbytes[prec]));
        BCK(upload(&bt->d_groups[prec], hg));
        BCK(upload(&bt->d_group_off[prec], hoff));
        BCK(upload(&bt->d_stream[prec], ent));
        BCK(upload(&bt->d_stream_off[prec], soff));
    }
    {   // low-rank (system, rhs) pairs, dealt round robin
        std::vector<std::vector<int32_t>> pb(grid);
        std::vector<int32_t> hpairs, hpoff(grid + 1, 0);
        int t = 0;
        for (int k = 0; k < nsys; ++k)
            if (bt->sx[k].r > 0)
                for (int j = 0; j < nr; ++j, ++t) {
                    pb[t % grid].push_back(k);
                    pb[t % grid].push_back(j);
                }
        for (int b = 0; b < grid; ++b) {
            hpoff[b] = (int32_t)(hpairs.size() / 2);
            hpairs.insert(hpairs.end(), pb[b].begin(), pb[b].end());
        }
        hpoff[grid] = (int32_t)(hpairs.size() / 2);
        BCK(upload(&bt->d_pairs, hpairs));
        BCK(upload(&bt->d_pair_off, hpoff));
    }
    // per-system scratch (sized in doubles; the FP32 form uses the front of each piece)
    std::vector<int64_t> so(nsys + 1, 0);
    auto al = [](int64_t x) { return (x + 31) / 32 * 32; };  // 256-byte pieces
    for (int k = 0; k < nsys; ++k) {
        const SysExport &e = bt->sx[k];
        so[k + 1] = so[k] + al((int64_t)nr * 2 * (e.q + 1)) + al((int64_t)nr * (e.q + 1)) +
                    al((int64_t)nr * e.s * std::max(e.r, 1)) + al((int64_t)nr * std::max(e.r, 1));
    }
    BCK(cudaMalloc(&bt->d_scratch, sizeof(double) * std::max<int64_t>(so[nsys], 1)));
    BCK(cudaMemset(bt->d_scratch, 0, sizeof(double) * std::max<int64_t>(so[nsys], 1)));
    std::vector<BatchSys<double>> s64(nsys);
    std::vector<BatchSys<float>> s32(nsys);
    double *sc = static_cast<double *>(bt->d_scratch);
    for (int k = 0; k < nsys; ++k) {
        const SysExport &e = bt->sx[k];
        double *w = sc + so[k];
        double *a = w + al((int64_t)nr * 2 * (e.q + 1));
        double *pt = a + al((int64_t)nr * (e.q + 1));
        double *d = pt + al((int64_t)nr * e.s * std::max(e.r, 1));
        auto fillsys = [&](auto &B, int prec, auto *tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            B.ioff = e.ioff;
            B.goff = e.goff;
            B.perm = e.perm;
            B.V = prec == 0 ? (const void *)e.V : (const void *)e.Vb;
            B.ldv = e.ldv;
            B.G = reinterpret_cast<const T *>(prec == 0 ? (const void *)e.G : (const void *)e.Gf);
            B.wbuf = reinterpret_cast<T *>(w);
            B.acc = reinterpret_cast<T *>(a);
            B.part = reinterpret_cast<T *>(pt);
            B.dco = reinterpret_cast<T *>(d);
            B.voff = bt->voff[k];
            B.n = e.n;
            B.s = e.s;
            B.p = e.p;
            B.q = e.q;
            B.r = e.r;
            B.m = e.m;
        };
        fillsys(s64[k], 0, (double *)nullptr);
        fillsys(s32[k], 1, (float *)nullptr);
    }
    {
        BatchSys<double> *p64 = nullptr;
        BatchSys<float> *p32 = nullptr;
        BCK(upload(&p64, s64));
        bt->d_sys[0] = p64;
        BCK(upload(&p32, s32));
        bt->d_sys[1] = p32;
    }
    BCK(cudaMalloc(&bt->d_bar, 16));
    BCK(cudaMemset(bt->d_bar, 0, 16));
    BCK(cudaMalloc(&bt->d_err, sizeof(int) * 2));
    BCK(cudaMemset(bt->d_err, 0, sizeof(int) * 2));

    // problems and chunks of the batched Krylov kernels
    std::vector<BkProb> probs;
    std::vector<BkChunk> chunks;
    for (int k = 0; k < nsys; ++k)
        for (int j = 0; j < nr; ++j) {
            BkProb p;
            p.off = bt->voff[k] + (int64_t)j * bt->sx[k].n;
            p.n = bt->sx[k].n;
            p.sys = k;
            p.nc = std::max(1, (p.n + bt->kchunk - 1) / bt->kchunk);
            p.c0 = (int32_t)chunks.size();
            for (int c = 0; c < p.nc; ++c) {
                BkChunk ch;
                ch.b = p.off + (int64_t)p.n * c / p.nc;
                ch.e = p.off + (int64_t)p.n * (c + 1) / p.nc;
                ch.prob = (int32_t)probs.size();
                ch.pad = 0;
                chunks.push_back(ch);
            }
            probs.push_back(p);
        }
    std::vector<BkSys> bs(nsys);
    for (int k = 0; k < nsys; ++k) {
        bs[k].rp = bt->sx[k].rp;
        bs[k].ci = bt->sx[k].ci;
        bs[k].av = bt->sx[k].av;
    }
    bt->nchunk = (int)chunks.size();
    bt->h_probs = probs;
    BCK(upload(&bt->d_chunks, chunks));
    BCK(upload(&bt->d_probs, probs));
    BCK(upload(&bt->d_bsys, bs));
    BCK(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
    return PSLR_OK;
}

// ------------------------------------------------------------------ apply

static pslr_status batch_check(pslr_batch *bt) {
    for (int k = 0; k < bt->nsys; ++k)
        if (sys_lr_gen(bt->ctx[k]) != bt->sx[k].lr_gen)
            return bfail(bt, PSLR_ERR_STATE,
                         "batch: the low-rank term of system %d was replaced after pslr_batch_create; "
                         "create the batch again", k);
    return PSLR_OK;
}

// form 0: FP64; 1: FP32 in and out; 2: FP32 arithmetic, FP64 in and out.
static pslr_status batch_launch(pslr_batch *bt, int form, const void *b, void *z, const int *skip,
                                const int *active, cudaStream_t st) {
    const int prec = form == 0 ? 0 : 1;
    auto fill = [&](auto &P) {
        P.segbase = bt->d_seg[prec];
        P.groups = bt->d_groups[prec];
        P.group_off = bt->d_group_off[prec];
        P.pairs = bt->d_pairs;
        P.pair_off = bt->d_pair_off;
        P.stream = bt->d_stream[prec];
        P.stream_off = bt->d_stream_off[prec];
        P.ring = bt->ring[prec];
        P.slot_bytes = bt->slot_bytes[prec];
        P.xs = bt->xs[prec];
        P.gs = bt->gs[prec];
        P.max_m = bt->max_m;
        P.nrhs = bt->nrhs;
        P.grid = bt->grid;
        P.any_lr = bt->any_lr;
        P.pair64 = bt->pair64;
        P.bar = bt->d_bar;
        P.err = bt->d_err;
        P.skip = skip;
        P.active = active;
        P.wait_limit = bt->wait_limit;
    };
    cudaError_t e;
    if (form == 0) {
        BatchParams<double, double> P;
        fill(P);
        P.sys = static_cast<const BatchSys<double> *>(bt->d_sys[0]);
        P.b = static_cast<const double *>(b);
        P.z = static_cast<double *>(z);
        e = launch_batch(0, &P, bt->smem[0], st);
    } else if (form == 1) {
        BatchParams<float, float> P;
        fill(P);
        P.sys = static_cast<const BatchSys<float> *>(bt->d_sys[1]);
        P.b = static_cast<const float *>(b);
        P.z = static_cast<float *>(z);
        e = launch_batch(1, &P, bt->smem[1], st);
    } else {
        BatchParams<float, double> P;
        fill(P);
        P.sys = static_cast<const BatchSys<float> *>(bt->d_sys[1]);
        P.b = static_cast<const double *>(b);
        P.z = static_cast<double *>(z);
        e = launch_batch(2, &P, bt->smem[1], st);
    }
    if (e != cudaSuccess) return bfail(bt, PSLR_ERR_CUDA, "batched apply launch: %s", cudaGetErrorString(e));
    return PSLR_OK;
}

// ------------------------------------------------------------------ FGMRES

static pslr_status krylov_ensure(pslr_batch *bt, int K) {
    if (bt->kK == K) return PSLR_OK;
    free_krylov(bt);
    const int64_t N = bt->n_total;
    const int P = bt->nprob, ldp = K + 1;
    BCK(cudaMalloc(&bt->d_V, sizeof(double) * (size_t)N * (K + 1)));
    BCK(cudaMalloc(&bt->d_Z, sizeof(double) * (size_t)N * K));
    BCK(cudaMemset(bt->d_V, 0, sizeof(double) * (size_t)N * (K + 1)));
    BCK(cudaMemset(bt->d_Z, 0, sizeof(double) * (size_t)N * K));
    BCK(cudaMalloc(&bt->d_w, sizeof(double) * (size_t)N));
    BCK(cudaMalloc(&bt->d_r, sizeof(double) * (size_t)N));
    BCK(cudaMalloc(&bt->d_b, sizeof(double) * (size_t)N));
    BCK(cudaMalloc(&bt->d_x, sizeof(double) * (size_t)N));
    // state: doubles first, then ints
    const size_t nd = 1 + (size_t)P * 4                      // rtol; bn, rn, hn, relres
                      + (size_t)P * ldp * K                  // H
                      + (size_t)P * 2 * K                    // rot
                      + (size_t)P * ldp * 3                  // gam, h1, h2
                      + (size_t)P * K                        // y
                      + (size_t)bt->nchunk * ldp * 2;        // pa, pb
    const size_t ni = (size_t)P * 4 + 3 + (size_t)bt->nsys;
    BCK(cudaMalloc(&bt->d_state, sizeof(double) * nd + sizeof(int) * ni));
    BCK(cudaMemset(bt->d_state, 0, sizeof(double) * nd + sizeof(int) * ni));
    double *d = static_cast<double *>(bt->d_state);
    BkState &S = bt->S;
    S.rtol = d; d += 1;
    S.bn = d; d += P;
    S.rn = d; d += P;
    S.hn = d; d += P;
    S.relres = d; d += P;
    S.H = d; d += (size_t)P * ldp * K;
    S.rot = d; d += (size_t)P * 2 * K;
    S.gam = d; d += (size_t)P * ldp;
    S.h1 = d; d += (size_t)P * ldp;
    S.h2 = d; d += (size_t)P * ldp;
    S.y = d; d += (size_t)P * K;
    S.pa = d; d += (size_t)bt->nchunk * ldp;
    S.pb = d; d += (size_t)bt->nchunk * ldp;
    int *ip = reinterpret_cast<int *>(d);
    S.stop = ip; ip += P;
    S.jd = ip; ip += P;
    S.conv = ip; ip += P;
    S.its = ip; ip += P;
    S.remaining = ip; ip += 1;
    S.skip = ip; ip += 1;
    S.maxit = ip; ip += 1;
    S.sys_active = ip;
    S.nsys = bt->nsys;
    S.nrhs = bt->nrhs;
    S.K = K;
    bt->kK = K;
    return PSLR_OK;
}

// One restart cycle: K Arnoldi steps (apply, CGS2, Givens, normalise), then
// least squares, x += Z y, the true residual and the restart decision.
static pslr_status enqueue_cycle(pslr_batch *bt, int form, cudaStream_t st) {
    const BkState &S = bt->S;
    const int K = S.K, nc = bt->nchunk, P = bt->nprob;
    const int64_t N = bt->n_total;
    for (int j = 0; j < K; ++j) {
        const double *vj = bt->d_V + (size_t)j * N;
        double *zj = bt->d_Z + (size_t)j * N;
        pslr_status a = batch_launch(bt, form, vj, zj, S.skip, S.sys_active, st);
        if (a != PSLR_OK) return a;
        bk_spmv_dots(nc, j, bt->d_chunks, bt->d_probs, bt->d_bsys, zj, bt->d_w, bt->d_V, N, S, st);
        bk_update(nc, j, bt->d_chunks, bt->d_probs, bt->d_w, bt->d_V, N, S.pa, S.pb, S.h1, 0, S, st);
        bk_update(nc, j, bt->d_chunks, bt->d_probs, bt->d_w, bt->d_V, N, S.pb, S.pa, S.h2, 1, S, st);
        bk_hessenberg(j, P, bt->d_probs, S, st);
        bk_normalize(nc, bt->d_chunks, bt->d_w, bt->d_V + (size_t)(j + 1) * N, S, st);
    }
    bk_lsq(P, S, st);
    bk_gemv_add(nc, bt->d_chunks, bt->d_Z, N, bt->d_x, S, st);
    bk_residual(nc, bt->d_chunks, bt->d_probs, bt->d_bsys, bt->d_x, bt->d_b, bt->d_r, S, st);
    bk_restart(0, P, bt->d_probs, S, st);
    bk_start(nc, bt->d_chunks, bt->d_r, bt->d_V, S, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(bt, PSLR_ERR_CUDA, "batched FGMRES launch: %s", cudaGetErrorString(e));
    return PSLR_OK;
}

// The cycle as a CUDA graph (captured on the batch's own stream), or nullptr
// when capture or instantiation is not available.
// Problems that still run when at most this many remain are finished on
// their own systems (pslr_solve): one single-system iteration per step
// instead of a whole batched step, and the systems in parallel.
constexpr int kHandoffProblems = 16;

// Finish the running problems on their own systems.  At a cycle boundary the
// restarted FGMRES of problem p depends only on its current residual r =
// b - A x (in d_r after the cycle end), so solving A e = r with the relative
// tolerance rtol ||b|| / ||r|| and adding e to x continues exactly the same
// iteration (the same Krylov spaces, the same stopping test rtol ||b||), up
// to rounding.  One host thread and stream per system: a system's problems
// run one after another (they share its context), different systems at once.
static pslr_status handoff(pslr_batch *bt, double rtol, int restart, int maxit, pslr_prec prec, cudaStream_t s) {
    const BkState &S = bt->S;
    const int P = bt->nprob;
    std::vector<int> conv(P), its(P);
    std::vector<double> bn(P), rn(P), rel(P);
    BCK(cudaMemcpyAsync(conv.data(), S.conv, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(its.data(), S.its, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(bn.data(), S.bn, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(rn.data(), S.rn, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(rel.data(), S.relres, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));  // also: d_r and d_x of the last cycle are complete
    std::map<int, std::vector<int>> by_sys;
    for (int p = 0; p < P; ++p)
        if (conv[p] == 0) by_sys[bt->h_probs[p].sys].push_back(p);
    if (bt->hstream.empty()) {
        bt->hstream.assign(bt->nsys, nullptr);
        bt->he.assign(bt->nsys, nullptr);
    }
    for (const auto &kv : by_sys) {
        const int k = kv.first;
        if (!bt->hstream[k]) BCK(cudaStreamCreateWithFlags(&bt->hstream[k], cudaStreamNonBlocking));
        if (!bt->he[k]) BCK(cudaMalloc(&bt->he[k], sizeof(double) * std::max(1, bt->sx[k].n)));
    }
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    struct Job {
        int sys;
        const std::vector<int> *probs;
        pslr_status status = PSLR_OK;
        int failed = -1;
    };
    std::vector<Job> jobs;
    for (const auto &kv : by_sys) jobs.push_back(Job{kv.first, &kv.second});
    auto work = [&](Job &J) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            J.status = PSLR_ERR_CUDA;
            return;
        }
        cudaStream_t hs = bt->hstream[J.sys];
        double *e = bt->he[J.sys];
        for (int p : *J.probs) {  // each p belongs to this job alone
            const BkProb &pr = bt->h_probs[p];
            int its2 = 0;
            double rel2 = 0.0;
            const pslr_status st = pslr_solve(bt->ctx[J.sys], bt->d_r + pr.off, e, rtol * bn[p] / rn[p], restart,
                                              maxit - its[p], prec, 0, &its2, &rel2, hs);
            if (st != PSLR_OK && st != PSLR_ERR_NOT_CONVERGED && st != PSLR_ERR_NAN) {
                J.status = st;
                J.failed = p;
                return;
            }
            if (st != PSLR_ERR_NAN) launch_axpy(pr.n, 1.0, e, bt->d_x + pr.off, hs);
            its[p] += its2;
            rel[p] = rel2 * rn[p] / bn[p];
            conv[p] = st == PSLR_OK ? 1 : (st == PSLR_ERR_NAN ? 3 : 2);
        }
        if (cudaStreamSynchronize(hs) != cudaSuccess) J.status = PSLR_ERR_CUDA;
    };
    if (jobs.size() == 1) {
        work(jobs[0]);
    } else {
        std::vector<std::thread> th;
        th.reserve(jobs.size());
        size_t started = 0;
        try {  // no exception may leave the C ABI: jobs without a thread run here
            for (; started < jobs.size(); ++started) th.emplace_back(work, std::ref(jobs[started]));
        } catch (...) {
        }
        for (size_t u = started; u < jobs.size(); ++u) work(jobs[u]);
        for (std::thread &t : th) t.join();
    }
    for (const Job &J : jobs) {
        if (J.status == PSLR_OK) continue;
        if (J.failed >= 0)
            return bfail(bt, J.status, "batch_solve: finishing problem %d on its system: %s", J.failed,
                         pslr_last_error(bt->ctx[J.sys]));
        return bfail(bt, J.status, "batch_solve: finishing problems on system %d: %s", J.sys,
                     cudaGetErrorString(cudaGetLastError()));
    }
    for (const Job &J : jobs) bt->handoff += (int)J.probs->size();
    BCK(cudaMemcpyAsync(S.conv, conv.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(S.its, its.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(S.relres, rel.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
    BCK(cudaStreamSynchronize(s));  // the host vectors above must outlive the copies
    return PSLR_OK;
}

static cudaGraphExec_t cycle_graph(pslr_batch *bt, int form) {
    const auto key = std::make_tuple(form, bt->S.K, bt->wait_limit);
    auto it = bt->graphs.find(key);
    if (it != bt->graphs.end()) return it->second;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    if (cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const pslr_status st = enqueue_cycle(bt, form, bt->cap);
    const cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
    if (st != PSLR_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) x = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (x) bt->graphs[key] = x;
    return x;
}

extern "C" {

pslr_status pslr_batch_create(int32_t nsys, pslr_ctx *const *systems, int32_t nrhs, int32_t group,
                              pslr_batch **out) {
    pslr_batch_opts o;
    std::memset(&o, 0, sizeof(o));
    o.group[0] = o.group[1] = group;
    o.pair_rhs = 1;
    return pslr_batch_create_opts(nsys, systems, nrhs, &o, out);
}

pslr_status pslr_batch_create_opts(int32_t nsys, pslr_ctx *const *systems, int32_t nrhs, const pslr_batch_opts *opts,
                                   pslr_batch **out) {
    TraceRange trace("pslr_batch_create");
    pslr_batch *bt = nullptr;
    if (out) *out = nullptr;
    const bool gok = opts && opts->group[0] >= 0 && opts->group[0] <= kMaxGroup && opts->group[1] >= 0 &&
                     opts->group[1] <= kMaxGroup;
    if (!out || nsys < 1 || !systems || nrhs < 1 || nrhs > kMaxBatchRhs || !gok)
        return bfail(nullptr, PSLR_ERR_ARG, "batch_create: bad argument (nsys >= 1, nrhs 1..%d, group 0..%d)",
                     kMaxBatchRhs, kMaxGroup);
    if (opts->ring_max[0] < 0 || opts->ring_max[1] < 0 || (opts->ring_max[0] > 0 && opts->ring_max[0] < 2) ||
        (opts->ring_max[1] > 0 && opts->ring_max[1] < 2) || opts->krylov_chunk < 0 ||
        (opts->krylov_chunk > 0 && (opts->krylov_chunk < 64 || opts->krylov_chunk > (1 << 20))) ||
        (opts->pair_rhs != 0 && opts->pair_rhs != 1))
        return bfail(nullptr, PSLR_ERR_ARG,
                     "batch_create: bad option (ring_max 0 or >= 2, krylov_chunk 0 or 64..2^20, pair_rhs 0 or 1)");
    std::vector<SysExport> sx(nsys);
    for (int k = 0; k < nsys; ++k) {
        if (!systems[k] || !sys_export(systems[k], &sx[k]))
            return bfail(nullptr, PSLR_ERR_ARG, "batch_create: system %d is not set up", k);
        if (sx[k].factor == 1)
            return bfail(nullptr, PSLR_ERR_ARG,
                         "batch_create: system %d uses exact LU factors; the batch takes ILU(0) and ILUT systems", k);
        if (sx[k].omega != 1.0)
            return bfail(nullptr, PSLR_ERR_STATE,
                         "batch_create: system %d applies the Neumann polynomial (pslr_set_neumann); the batch "
                         "applies PSLR", k);
        if (sx[k].r > 0 && (!sx[k].V || !sx[k].Vb || !sx[k].G || !sx[k].Gf))
            return bfail(nullptr, PSLR_ERR_STATE, "batch_create: system %d has no low-rank term on the device", k);
    }
    bt = new pslr_batch();
    bt->nsys = nsys;
    bt->nrhs = nrhs;
    bt->group_req[0] = opts->group[0];
    bt->group_req[1] = opts->group[1];
    bt->ring_max[0] = opts->ring_max[0];
    bt->ring_max[1] = opts->ring_max[1];
    bt->kchunk = opts->krylov_chunk > 0 ? opts->krylov_chunk : kBkChunk;
    bt->pair64 = opts->pair_rhs;
    bt->ctx.assign(systems, systems + nsys);
    bt->sx = sx;
    pslr_status st = batch_build(bt);
    if (st != PSLR_OK) {
        g_create_error = bt->err;
        free_batch(bt);
        delete bt;
        return st;
    }
    *out = bt;
    return PSLR_OK;
}

pslr_status pslr_batch_apply(pslr_batch *bt, const void *b_dev, void *z_dev, pslr_prec prec, void *stream) {
    if (!bt || !b_dev || !z_dev || (prec != PSLR_FP64 && prec != PSLR_FP32))
        return bfail(bt, PSLR_ERR_ARG, "batch_apply: bad argument");
    pslr_status st = batch_check(bt);
    if (st != PSLR_OK) return st;
    return batch_launch(bt, prec == PSLR_FP64 ? 0 : 1, b_dev, z_dev, nullptr, nullptr,
                        static_cast<cudaStream_t>(stream));
}

pslr_status pslr_batch_sync(pslr_batch *bt, void *stream) {
    if (!bt) return PSLR_ERR_ARG;
    BCK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int err = 0;
    BCK(cudaMemcpy(&err, bt->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) {
        BCK(cudaMemset(bt->d_err, 0, sizeof(int) * 2));
        BCK(cudaMemset(bt->d_bar, 0, 16));
        return bfail(bt, (pslr_status)err, "batch: a device-side wait gave up (status %d)", err);
    }
    return PSLR_OK;
}

pslr_status pslr_batch_solve(pslr_batch *bt, const double *b_dev, double *x_dev, double rtol, int32_t restart,
                             int32_t maxit, pslr_prec prec, int32_t *iters, double *relres, void *stream) {
    TraceRange trace("pslr_batch_solve");
    if (!bt || !b_dev || !x_dev || restart < 1 || restart > 127 || maxit < 0 || !(rtol > 0.0) ||
        (prec != PSLR_FP64 && prec != PSLR_FP32))
        return bfail(bt, PSLR_ERR_ARG, "batch_solve: bad argument (restart must be 1..127)");
    pslr_status st = batch_check(bt);
    if (st != PSLR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = krylov_ensure(bt, restart);
    if (st != PSLR_OK) return st;
    const BkState &S = bt->S;
    BCK(cudaMemcpyAsync(const_cast<double *>(S.rtol), &rtol, sizeof(double), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(const_cast<int *>(S.maxit), &maxit, sizeof(int), cudaMemcpyHostToDevice, s));
    const int P = bt->nprob, nc = bt->nchunk;
    const int64_t N = bt->n_total;
    const int form = prec == PSLR_FP64 ? 0 : 2;
    BCK(cudaMemcpyAsync(bt->d_b, b_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    BCK(cudaMemsetAsync(bt->d_x, 0, sizeof(double) * N, s));
    BCK(cudaMemsetAsync(S.conv, 0, sizeof(int) * P, s));
    bk_residual(nc, bt->d_chunks, bt->d_probs, bt->d_bsys, nullptr, bt->d_b, bt->d_r, S, s);
    bk_restart(1, P, bt->d_probs, S, s);
    bk_start(nc, bt->d_chunks, bt->d_r, bt->d_V, S, s);
    int remaining = 0;
    BCK(cudaMemcpyAsync(&remaining, S.remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    cudaGraphExec_t g = remaining > 0 ? cycle_graph(bt, form) : nullptr;
    bt->graph_used = g != nullptr;
    bt->handoff = 0;
    for (int cyc = 0; remaining > 0 && cyc <= maxit; ++cyc) {
        if (g) {
            BCK(cudaGraphLaunch(g, s));
        } else {
            st = enqueue_cycle(bt, form, s);
            if (st != PSLR_OK) return st;
        }
        BCK(cudaMemcpyAsync(&remaining, S.remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
        st = pslr_batch_sync(bt, stream);
        if (st != PSLR_OK) return st;
        if (remaining > 0 && remaining <= kHandoffProblems && P > kHandoffProblems) {
            st = handoff(bt, rtol, restart, maxit, prec, s);
            if (st != PSLR_OK) return st;
            remaining = 0;
        }
    }
    BCK(cudaMemcpyAsync(x_dev, bt->d_x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    std::vector<int> conv(P), its(P);
    std::vector<double> rel(P);
    BCK(cudaMemcpyAsync(conv.data(), S.conv, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(its.data(), S.its, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(rel.data(), S.relres, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (iters) std::copy(its.begin(), its.end(), iters);
    if (relres) std::copy(rel.begin(), rel.end(), relres);
    int nan = 0, nconv = 0;
    for (int p = 0; p < P; ++p) {
        nan += conv[p] == 3;
        nconv += conv[p] == 1;
    }
    if (nan) return bfail(bt, PSLR_ERR_NAN, "batch_solve: %d problem(s) went non-finite", nan);
    if (nconv < P)
        return bfail(bt, PSLR_ERR_NOT_CONVERGED, "batch_solve: %d of %d problems reached maxit = %d", P - nconv, P,
                     maxit);
    return PSLR_OK;
}

pslr_status pslr_batch_get_info(const pslr_batch *bt, pslr_batch_info *info) {
    if (!bt || !info) return PSLR_ERR_ARG;
    info->nsys = bt->nsys;
    info->nrhs = bt->nrhs;
    info->nprob = bt->nprob;
    info->n_total = bt->n_total;
    info->items = bt->items;
    info->grid = bt->grid;
    info->ring[0] = bt->ring[0];
    info->ring[1] = bt->ring[1];
    info->group[0] = bt->group[0];
    info->group[1] = bt->group[1];
    info->groups[0] = bt->ngroups[0];
    info->groups[1] = bt->ngroups[1];
    info->max_m = bt->max_m;
    info->max_p = bt->max_p;
    info->max_q = bt->max_q;
    info->apply_bytes_fp64 = bt->apply_bytes[0];
    info->apply_bytes_fp32 = bt->apply_bytes[1];
    info->graph = bt->graph_used;
    info->handoff = bt->handoff;
    info->krylov_chunk = bt->kchunk;
    info->pair_rhs = bt->pair64;
    return PSLR_OK;
}

int64_t pslr_batch_set_wait_limit(pslr_batch *bt, int64_t polls) {
    if (!bt) return -1;
    const int64_t old = bt->wait_limit;
    bt->wait_limit = polls;
    return old;
}

const char *pslr_batch_last_error(const pslr_batch *bt) {
    return bt ? bt->err.c_str() : g_create_error.c_str();
}

void pslr_batch_destroy(pslr_batch *bt) {
    if (!bt) return;
    cudaDeviceSynchronize();
    free_batch(bt);
    delete bt;
}

}  // extern "C"
