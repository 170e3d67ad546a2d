// Host side of libpslr: set-up (Section 2 reordering, Algorithm 1 local
// factors), device layout, and the C ABI of include/pslr.h.
//
// The set-up is plain C++ on the host (it is not part of the timed apply):
// geometric partition, interface detection, the [interior by subdomain |
// interface by subdomain] permutation, the per-subdomain blocks B_i, E_i, F_i,
// C_i and the rows of C_g, ILU(0) or dense pivoted LU of every B_i and C_i,
// level scheduling of the triangular factors, and packing into the segment
// layout described in pslr_internal.h, for the forward and transposed
// directions and for FP64 and FP32 values.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "pslr.h"
#include "pslr_internal.h"
#include "pslr_sys.h"
#include "pslr_trace.h"

namespace pslr {
// kernels (pslr_apply.cu, pslr_krylov.cu)
cudaError_t launch_apply_fp64(const ApplyParams<double> &P, int smem, bool dual, bool merged, cudaStream_t st);
cudaError_t launch_apply_fp32(const ApplyParams<float> &P, int smem, bool dual, bool merged, cudaStream_t st);
cudaError_t launch_apply_f32d(const ApplyParams<float, double> &P, int smem, bool dual, bool merged,
                              cudaStream_t st);
cudaError_t launch_err_fp64(const ErrParams<double> &P, int smem, bool dual, bool merged, cudaStream_t st);

// The persistent kernels' launchers set the kernel's dynamic shared-memory
// limit and then launch; contexts applied from several host threads at once
// (the batched solve finishing problems on their systems) must not interleave
// these two steps, or one launch can meet another context's smaller limit.
static std::mutex g_launch_mutex;
int max_coresident_apply(int smem, bool fp32, bool dual, bool merged);
cudaError_t launch_apply_fp64_unit(const ApplyParams<double> &P, int smem, bool dual, bool merged, cudaStream_t st);
// device ILU(0) of a block-diagonal matrix (pslr_ilu0.cu)
pslr_status ilu0_device_blocks(int n, int nb, const int32_t *bptr, const int32_t *rp, const int32_t *ci,
                               double *val_dev, cudaStream_t st, float *kernel_ms, int *bad_row, std::string &why);
int krylov_blocks(int n);
size_t krylov_part_doubles(int nblk, int nres);
int krylov_tickets();
void launch_cgs_pass(int n, int k, const double *V, int64_t ld, double *w, const double *hsub, int norm,
                     double *part, double *res, unsigned *ticket, const int32_t *rp, const int32_t *ci,
                     const double *av, const double *z, const int *skip, cudaStream_t st);
void launch_hess_normalize(int j, const double *h1, const double *h2, const double *wn2, double *H, int ldh,
                           double *rot, double *gam, const double *tol_abs, int *state, int *skip, int n,
                           const double *w, double *v, cudaStream_t st);
void launch_normalize(int n, const double *w, double *v, const double *hn, const int *skip,
                      cudaStream_t st);
void launch_gemv_add(int n, int k, const double *Z, int64_t ld, const double *y, double *x,
                     cudaStream_t st);
void launch_residual(int n, const int32_t *rp, const int32_t *ci, const double *av, const double *x,
                     const double *b, double *r, cudaStream_t st);
void launch_splitmix(int n, uint64_t seed, uint64_t j0, double *v, cudaStream_t st);
void launch_grad_values(int n, const int32_t *rp, const int32_t *ci, const double *lambda, const double *u,
                        double *g, cudaStream_t st);
}  // namespace pslr

using namespace pslr;

namespace pslr_part {
bool graph_partition(int n, const int32_t *rowptr, const int32_t *colind, int nparts, int32_t *part, int threads);
}

namespace {

// ---------------------------------------------------------------- utilities

struct Csr {  // local sparse block, columns ascending in each row
    int nr = 0, nc = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> v;
};

struct Row {  // one row of a segment: output row, off-diagonal entries, diagonal
    int row;
    std::vector<std::pair<int32_t, double>> e;
    double diag;
};

uint16_t f32_to_bf16(float f) {  // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

// Host record of one packed segment.
struct SegDesc {
    int64_t off;
    int32_t bytes;
};

// Segments of one direction and one precision, accumulated on the host.
struct SegStore {
    std::vector<char> bytes;
    std::vector<SegDesc> desc;
    int max_bytes = 0;
};

// Run f(0) .. f(n-1) on up to `threads` host threads (the calling thread
// included), indices handed out in increasing order.  f must only write state
// owned by its index.  Returns false if some f threw (the remaining indices
// still run); a pool that cannot be started runs the rest on this thread.
template <class F>
bool parallel_for(int n, int threads, F &&f) {
    std::atomic<int> next{0};
    std::atomic<bool> ok{true};
    auto work = [&]() {
        for (int i; (i = next.fetch_add(1)) < n;) {
            try {
                f(i);
            } catch (...) {
                ok = false;
            }
        }
    };
    std::vector<std::thread> pool;
    const int t = std::max(1, std::min(threads, n));
    try {
        for (int k = 1; k < t; ++k) pool.emplace_back(work);
    } catch (...) {
    }
    work();
    for (auto &th : pool) th.join();
    return ok;
}

// FNV-1a with the 64-bit prime, taken over 8-byte little-endian words (the
// tail byte by byte), continuing from h.
uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w = 0;
        for (int k = 0; k < 8; ++k) w |= (uint64_t)b[i + k] << (8 * k);
        h ^= w;
        h *= 0x100000001b3ull;
    }
    for (; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// pad128: the block's size is rounded up to 128 bytes (levels of a sweep, so
// that every level block of a multi-level segment starts on a 128-byte row of
// shared memory, as a slot does: the warps' record loads then touch no more
// rows than they must).
template <class T, class IDX>
void pack_segment(SegStore &S, const std::vector<Row> &rows, size_t b, size_t e, bool diag, int zero_col,
                  bool pad128) {
    int n = (int)(e - b), w = 0;
    for (size_t i = b; i < e; ++i) w = std::max<int>(w, (int)rows[i].e.size());
    const int np = seg_npad(n);
    const int64_t nbytes = pad128 ? align_up((int)seg_bytes<T, IDX>(n, w, diag), 128) : seg_bytes<T, IDX>(n, w, diag);
    SegDesc d;
    d.off = (int64_t)S.bytes.size();
    d.bytes = (int32_t)nbytes;
    S.bytes.resize(S.bytes.size() + nbytes, 0);
    char *base = S.bytes.data() + d.off;
    SegHdr h;
    std::memset(&h, 0, sizeof(h));
    h.n = (uint16_t)n;
    h.w = (uint8_t)w;
    h.flags = (uint8_t)((diag ? (unsigned)kSegDiag : 0u) | (sizeof(IDX) == 4 ? (unsigned)kSegGlobalCols : 0u));
    h.np = (uint16_t)np;
    const int fmt = seg_fmt_for(w);
    h.fmt = (uint8_t)fmt;
    if (fmt != kTile) h.w = (uint8_t)fmt;
    h.bytes = (uint32_t)nbytes;
    std::memcpy(base, &h, sizeof(h));
    base += sizeof(SegHdr);
    if (fmt != kTile) {
        const int K = fmt;
        IDX *idx = reinterpret_cast<IDX *>(base);
        T *val = reinterpret_cast<T *>(base + (size_t)np * rec_idx_bytes<IDX>(K));
        for (int j = 0; j < np; ++j) {
            const bool real = j < n;
            const Row *R = real ? &rows[b + j] : nullptr;
            IDX *ir = idx + (size_t)j * (K + 1);
            T *vr = val + (size_t)j * (K + 1);
            ir[0] = real ? (IDX)R->row : (IDX)0;
            for (int k = 0; k < K; ++k) {
                const bool has = real && k < (int)R->e.size();
                ir[1 + k] = has ? (IDX)R->e[k].first : (IDX)zero_col;
                vr[k] = has ? (T)R->e[k].second : T(0);
            }
            vr[K] = (real && diag) ? (T)(1.0 / R->diag) : T(1);  // rows without a diagonal scale by 1
        }
        S.max_bytes = std::max<int>(S.max_bytes, (int)nbytes);
        S.desc.push_back(d);
        return;
    }
    T *vals = reinterpret_cast<T *>(base);
    T *dinv = reinterpret_cast<T *>(base + (size_t)np * w * sizeof(T));
    IDX *cols = reinterpret_cast<IDX *>(base + (size_t)np * w * sizeof(T) + (diag ? np * sizeof(T) : 0));
    uint16_t *rws = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(cols) + (size_t)np * w * sizeof(IDX));
    for (int j = 0; j < np; ++j) {
        const bool real = j < n;
        const Row *R = real ? &rows[b + j] : nullptr;
        for (int k = 0; k < w; ++k) {
            const bool has = real && k < (int)R->e.size();
            vals[(size_t)k * np + j] = has ? (T)R->e[k].second : T(0);
            cols[(size_t)k * np + j] = has ? (IDX)R->e[k].first : (IDX)zero_col;
        }
        if (diag) dinv[j] = real ? (T)(1.0 / R->diag) : T(0);
        rws[j] = real ? (uint16_t)R->row : (uint16_t)0;
    }
    S.max_bytes = std::max<int>(S.max_bytes, (int)nbytes);
    S.desc.push_back(d);
}

// Split a row list into segments within kSegBudget bytes / kSegMaxRows rows.
// Returns the number of segments appended (an empty list appends none).
template <class T, class IDX>
int pack_rows(SegStore &S, const std::vector<Row> &rows, bool diag, int zero_col, bool pad128 = false) {
    int cnt = 0;
    size_t b = 0;
    while (b < rows.size()) {
        size_t e = b;
        int w = 0;
        while (e < rows.size() && (int)(e - b) < kSegMaxRows) {
            int w2 = std::max<int>(w, (int)rows[e].e.size());
            if (e > b && align_up((int)seg_bytes<T, IDX>((int)(e - b + 1), w2, diag), pad128 ? 128 : 1) > kSegBudget)
                break;
            w = w2;
            ++e;
        }
        pack_segment<T, IDX>(S, rows, b, e, diag, zero_col, pad128);
        ++cnt;
        b = e;
    }
    return cnt;
}

// Merge the one-level segments S.desc[d0..] of a sweep, which lie back to
// back in the store, into segments of consecutive levels of at most `budget`
// bytes (every block but a segment's last flagged kSegMore).  Returns the
// number of segments.
int merge_levels(SegStore &S, size_t d0, int budget) {
    std::vector<SegDesc> out;
    for (size_t d = d0; d < S.desc.size();) {
        SegDesc c = S.desc[d];
        size_t e = d + 1;
        while (e < S.desc.size() && c.bytes + S.desc[e].bytes <= budget &&
               S.desc[e].off == S.desc[e - 1].off + S.desc[e - 1].bytes) {
            S.bytes[(size_t)S.desc[e - 1].off + offsetof(SegHdr, flags)] |= (char)kSegMore;
            c.bytes += S.desc[e].bytes;
            ++e;
        }
        S.max_bytes = std::max<int>(S.max_bytes, c.bytes);
        out.push_back(c);
        d = e;
    }
    S.desc.resize(d0);
    S.desc.insert(S.desc.end(), out.begin(), out.end());
    return (int)out.size();
}

// Level schedule of a triangular sweep: lower (deps on smaller columns,
// processed 0..n-1) or upper (deps on larger columns, processed n-1..0).
// Returns the rows of every level, levels in dependency order.
std::vector<std::vector<int>> levels(const Csr &T, bool lower) {
    int n = T.nr;
    std::vector<int> lev(n, 0);
    int maxl = -1;
    for (int t = 0; t < n; ++t) {
        int r = lower ? t : n - 1 - t;
        int l = 0;
        for (int k = T.rp[r]; k < T.rp[r + 1]; ++k) {
            int c = T.ci[k];
            if ((lower && c < r) || (!lower && c > r)) l = std::max(l, lev[c] + 1);
        }
        lev[r] = l;
        maxl = std::max(maxl, l);
    }
    std::vector<std::vector<int>> L(maxl + 1);
    for (int r = 0; r < n; ++r) L[lev[r]].push_back(r);
    return L;
}

// Rows of a triangular sweep level: off-diagonal entries of T in the row and
// (with_diag) its diagonal.
std::vector<Row> sweep_rows(const Csr &T, const std::vector<int> &lv, bool lower, bool with_diag) {
    std::vector<Row> rows;
    rows.reserve(lv.size());
    for (int r : lv) {
        Row R;
        R.row = r;
        R.diag = 1.0;
        for (int k = T.rp[r]; k < T.rp[r + 1]; ++k) {
            int c = T.ci[k];
            if (c == r) R.diag = T.v[k];
            else if ((lower && c < r) || (!lower && c > r)) R.e.push_back({c, T.v[k]});
        }
        if (!with_diag) R.diag = 1.0;
        rows.push_back(std::move(R));
    }
    return rows;
}

Csr transpose(const Csr &A) {
    Csr T;
    T.nr = A.nc;
    T.nc = A.nr;
    T.rp.assign(T.nr + 1, 0);
    for (int k = 0; k < (int)A.ci.size(); ++k) T.rp[A.ci[k] + 1]++;
    for (int i = 0; i < T.nr; ++i) T.rp[i + 1] += T.rp[i];
    T.ci.resize(A.ci.size());
    T.v.resize(A.v.size());
    std::vector<int32_t> pos(T.rp.begin(), T.rp.end() - 1);
    for (int r = 0; r < A.nr; ++r)
        for (int k = A.rp[r]; k < A.rp[r + 1]; ++k) {
            int p = pos[A.ci[k]]++;
            T.ci[p] = r;
            T.v[p] = A.v[k];
        }
    return T;
}

// Rows of an ELL block (all rows with at least one entry).
std::vector<Row> ell_rows(const Csr &A) {
    std::vector<Row> rows;
    for (int r = 0; r < A.nr; ++r) {
        if (A.rp[r + 1] == A.rp[r]) continue;
        Row R;
        R.row = r;
        R.diag = 1.0;
        for (int k = A.rp[r]; k < A.rp[r + 1]; ++k) R.e.push_back({A.ci[k], A.v[k]});
        rows.push_back(std::move(R));
    }
    return rows;
}

// ILU(0) of a local block in place (IKJ order, natural ordering, no
// pivoting): strictly lower part becomes L (unit diagonal), the rest U.
bool ilu0_inplace(Csr &M) {
    const int n = M.nr;
    std::vector<int> dpos(n, -1), where(n, -1);
    for (int i = 0; i < n; ++i)
        for (int k = M.rp[i]; k < M.rp[i + 1]; ++k)
            if (M.ci[k] == i) dpos[i] = k;
    for (int i = 0; i < n; ++i) {
        if (dpos[i] < 0) return false;
        for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) where[M.ci[k]] = k;
        for (int k = M.rp[i]; k < dpos[i]; ++k) {
            const int j = M.ci[k];
            const double piv = M.v[dpos[j]];
            if (piv == 0.0) return false;
            const double l = M.v[k] / piv;
            M.v[k] = l;
            for (int t = dpos[j] + 1; t < M.rp[j + 1]; ++t) {
                const int w = where[M.ci[t]];
                if (w >= 0) M.v[w] -= l * M.v[t];
            }
        }
        if (M.v[dpos[i]] == 0.0) return false;
        for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) where[M.ci[k]] = -1;
    }
    return true;
}

// Dense LU with partial pivoting (largest |a|, first on ties) of a local
// block; returns L (unit diagonal implied, strictly lower) and U (upper with
// diagonal) as one combined sparse factor, and the row order piv: the
// factored matrix is B(piv, :), i.e. (P b)_r = b[piv[r]].
bool dense_lu(const Csr &M, Csr &LU, std::vector<uint16_t> &piv) {
    const int n = M.nr;
    std::vector<double> a((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) a[(size_t)i * n + M.ci[k]] = M.v[k];
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
        int pr = k;
        double best = std::fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = std::fabs(a[(size_t)i * n + k]);
            if (v > best) {
                best = v;
                pr = i;
            }
        }
        if (best == 0.0) return false;
        if (pr != k) {
            for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)pr * n + j]);
            std::swap(perm[k], perm[pr]);
        }
        const double d = a[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double &l = a[(size_t)i * n + k];
            if (l == 0.0) continue;
            l /= d;
            for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    LU.nr = LU.nc = n;
    LU.rp.assign(n + 1, 0);
    LU.ci.clear();
    LU.v.clear();
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double v = a[(size_t)i * n + j];
            if (v != 0.0 || j == i) {
                LU.ci.push_back(j);
                LU.v.push_back(v);
            }
        }
        LU.rp[i + 1] = (int32_t)LU.ci.size();
    }
    piv.resize(n);
    for (int i = 0; i < n; ++i) piv[i] = (uint16_t)perm[i];
    return true;
}

// ILUT(tau) of a local block with no fill limit (the threshold incomplete LU
// the paper's Section 4 runs use, drop threshold 1e-2; Saad, Iterative
// Methods, Sec. 10.4, with the row scale of Saad's SPARSKIT ilut): the drop
// tolerance of row i is tol_i = tau * (sum_j |a_ij|) / nnz(a_i), the mean
// modulus of the block row (summed in stored column order).  Row i starts as
// a_i; for k < i in increasing order with w_k != 0, w_k <- w_k / u_kk,
// dropped if |w_k| < tol_i, else w <- w - w_k u_k (the upper part of row k,
// diagonal excluded); then every entry but the diagonal below tol_i is
// dropped.  The result is L
// (strictly lower, unit diagonal implied) and U (with diagonal) in one CSR,
// columns ascending.  false on a zero pivot.
bool ilut(const Csr &M, double tau, Csr &out) {
    const int n = M.nr;
    out.nr = out.nc = n;
    out.rp.assign(1, 0);
    out.ci.clear();
    out.v.clear();
    std::vector<double> w(n, 0.0);
    std::vector<char> nz(n, 0);
    std::vector<int32_t> diagpos(n, -1), cols;
    for (int i = 0; i < n; ++i) {
        double s1 = 0.0;
        for (int t = M.rp[i]; t < M.rp[i + 1]; ++t) s1 += std::fabs(M.v[t]);
        const int len = M.rp[i + 1] - M.rp[i];
        const double tol = len > 0 ? tau * (s1 / len) : 0.0;
        cols.clear();
        int lo = i;
        for (int t = M.rp[i]; t < M.rp[i + 1]; ++t) {
            const int j = M.ci[t];
            w[j] = M.v[t];
            nz[j] = 1;
            cols.push_back(j);
            lo = std::min(lo, j);
        }
        for (int k = lo; k < i; ++k) {
            if (!nz[k]) continue;
            const double wk = w[k] / out.v[diagpos[k]];
            if (std::fabs(wk) < tol) {
                w[k] = 0.0;
                nz[k] = 2;  // dropped: not kept, not used
                continue;
            }
            w[k] = wk;
            for (int t = diagpos[k] + 1; t < out.rp[k + 1]; ++t) {
                const int j = out.ci[t];
                if (!nz[j]) {
                    nz[j] = 1;
                    w[j] = 0.0;
                    cols.push_back(j);
                }
                w[j] -= wk * out.v[t];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int j : cols) {
            const bool keep = nz[j] == 1 && (j == i || std::fabs(w[j]) >= tol);
            if (keep) {
                if (j == i) diagpos[i] = (int32_t)out.ci.size();
                out.ci.push_back(j);
                out.v.push_back(w[j]);
            }
            w[j] = 0.0;
            nz[j] = 0;
        }
        out.rp.push_back((int32_t)out.ci.size());
        if (diagpos[i] < 0 || out.v[diagpos[i]] == 0.0 || !std::isfinite(out.v[diagpos[i]])) return false;
    }
    return true;
}

// Split the combined factor into L (strictly lower entries) and U.
void split_lu(const Csr &LU, Csr &Lo, Csr &Up) {
    Lo.nr = Lo.nc = Up.nr = Up.nc = LU.nr;
    Lo.rp.assign(LU.nr + 1, 0);
    Up.rp.assign(LU.nr + 1, 0);
    Lo.ci.clear(); Lo.v.clear(); Up.ci.clear(); Up.v.clear();
    for (int i = 0; i < LU.nr; ++i) {
        for (int k = LU.rp[i]; k < LU.rp[i + 1]; ++k) {
            if (LU.ci[k] < i) {
                Lo.ci.push_back(LU.ci[k]);
                Lo.v.push_back(LU.v[k]);
            } else {
                Up.ci.push_back(LU.ci[k]);
                Up.v.push_back(LU.v[k]);
            }
        }
        Lo.rp[i + 1] = (int32_t)Lo.ci.size();
        Up.rp[i + 1] = (int32_t)Up.ci.size();
    }
}

template <class X>
cudaError_t upload(X **dst, const std::vector<X> &src) {
    *dst = nullptr;
    size_t bytes = std::max<size_t>(src.size() * sizeof(X), 16);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

// ------------------------------------------------------------------ context

// A CTA-ordered segment stream on the device (see pslr_internal.h).
struct StreamDev {
    StreamEnt *ent = nullptr;
    int64_t *off = nullptr;
};

struct OpSetHost {
    char *seg = nullptr;                 // device: all segments
    int32_t *cnt = nullptr;              // device: kNCnt*s segment counts
    std::vector<SegDesc> hdesc;          // host: segment offsets/sizes
    std::vector<int32_t> hsub, hcnt;     // host: first descriptor and counts per subdomain
    int slot_bytes = 0;
    int ring = 0;
    int64_t seg_total = 0;
    int64_t cat_bytes[kNCnt] = {0, 0, 0, 0, 0, 0, 0};  // segment bytes per category, all subdomains
    int smem = 0;
    int grid = 0;
    bool dual = false;                   // two CTAs per SM (more subdomains than SMs)
    bool merged = false;                 // sweep segments hold several levels
    std::map<std::string, StreamDev> streams;  // keyed by launch shape
};

// Krylov workspace for vectors of length len and up to kcols basis columns:
// Gram-Schmidt partial sums, coefficients, norms and reduction tickets.
struct KWork {
    double *part = nullptr, *h1 = nullptr, *h2 = nullptr, *wn2 = nullptr, *hn = nullptr;
    unsigned *ticket = nullptr;
    int nblk = 0;
};

struct pslr_ctx {
    int n = 0, s = 0, p = 0, q = 0, factor = 0;
    int device_factor = 0;   // ILU(0) factors computed on the GPU
    float factor_ms = 0.f;   // time of that factorization kernel
    int rs = 8;              // column stride of the kernels' low-rank scratch (red_stride(r))
    double drop_tol = 0.0;  // ILUT threshold (factor 2)
    uint64_t seed = 0;
    std::vector<int32_t> part, iface, perm, ioff, goff;
    int max_p = 0, max_q = 0, levels_B = 0, levels_C = 0;
    int64_t nnz_A = 0, nnz_ilu = 0;
    int64_t nnz_blk[5] = {0, 0, 0, 0, 0};  // local factors of B and C0 (L+U), E, F, C_g
    int threads = 1;            // host threads of the set-up
    uint64_t layout_hash = 0;   // pslr_plan: hash of the packed device layout
    int64_t layout_errors = 0;  // pslr_plan: violations found by check_layout
    std::vector<int32_t> h_rp, h_ci;
    std::vector<double> h_av;
    // device: maps and matrices
    int32_t *d_perm = nullptr, *d_ioff = nullptr, *d_goff = nullptr;
    uint16_t *d_bpiv = nullptr, *d_cpiv = nullptr;
    OpSetHost ops[2][2];  // [direction: 0 forward, 1 transposed][precision]
    // forward FP64 applies without row pivots: the unit-diagonal operator set
    // (E rows and both sweeps scaled, see unit_rows) and the inverse U
    // diagonals by which the kernel scales the other solve right-hand sides
    bool has_unit = false;
    OpSetHost ops_unit;
    std::vector<double> h_dB, h_dC;
    double *d_dB = nullptr, *d_dC = nullptr;
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_rpT = nullptr, *d_ciT = nullptr;
    double *d_av = nullptr, *d_avT = nullptr;
    // low-rank term
    int m = 0, r = 0;
    uint64_t lr_gen = 0;         // incremented whenever the low-rank term is replaced
    double omega = 1.0;          // 1: PSLR; otherwise the Sec. 1 Neumann polynomial (pslr_set_neumann)
    int merge_levels = 0;        // pslr_opts::merge_levels
    std::vector<double> V, H, G;
    double *d_V = nullptr;       // q x r FP64 (leading dimension q)
    // the copies the apply reads: row-major, row stride ldv = r rounded up to 8, zero padded
    int ldv = 0;
    double *d_Vr = nullptr;      // FP64
    uint16_t *d_Vb = nullptr;    // BF16
    double *d_G = nullptr, *d_GT = nullptr;
    float *d_Gf = nullptr, *d_GTf = nullptr;
    // apply scratch
    double *d_wbuf = nullptr, *d_acc = nullptr, *d_part = nullptr;
    unsigned *d_bar = nullptr;
    int *d_err = nullptr;
    long long wait_limit = 1ll << 22;
    // Krylov workspace (allocated on demand) and the captured restart cycles
    int kr_restart = 0;
    KWork kw;
    double *d_ktol = nullptr;  // FGMRES absolute tolerance rtol ||b||
    cudaStream_t kcap = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> kgraphs;  // keyed by (precision, direction)
    double *d_kV = nullptr, *d_kZ = nullptr, *d_kw = nullptr, *d_kr = nullptr, *d_kH = nullptr;
    double *d_krot = nullptr, *d_kgam = nullptr;
    int *d_kstate = nullptr, *d_kskip = nullptr;
    double *d_eab = nullptr;  // E_rr scratch 2(q+1)
    void *d_io_b = nullptr, *d_io_z = nullptr;  // pslr_apply_host staging
    size_t io_bytes = 0;
    int *h_err = nullptr;  // pinned host copy of the error word (pslr_sync)
    std::string err;
};

namespace {

pslr_status fail(pslr_ctx *c, pslr_status st, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(c, PSLR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void cfree(void *p) {
    if (p) cudaFree(p);
}

void free_opset(OpSetHost &o) {
    cfree(o.seg);
    cfree(o.cnt);
    for (auto &kv : o.streams) {
        cfree(kv.second.ent);
        cfree(kv.second.off);
    }
    o = OpSetHost();
}

// The captured FGMRES cycles hold the apply's launch parameters (low-rank
// pointers, wait limit) and the Krylov workspace: drop them whenever either
// changes.
void drop_graphs(pslr_ctx *c) {
    for (auto &kv : c->kgraphs) cudaGraphExecDestroy(kv.second);
    c->kgraphs.clear();
}

void free_krylov(pslr_ctx *c) {
    drop_graphs(c);
    KWork &W = c->kw;
    for (void *p : {(void *)c->d_kV, (void *)c->d_kZ, (void *)c->d_kw, (void *)c->d_kr, (void *)c->d_kH,
                    (void *)c->d_krot, (void *)c->d_kgam, (void *)c->d_kstate, (void *)c->d_kskip,
                    (void *)c->d_ktol, (void *)W.part, (void *)W.h1,
                    (void *)W.h2, (void *)W.wn2, (void *)W.hn, (void *)W.ticket})
        cfree(p);
    c->d_kV = c->d_kZ = c->d_kw = c->d_kr = c->d_kH = c->d_krot = c->d_kgam = nullptr;
    c->d_kstate = c->d_kskip = nullptr;
    c->d_ktol = nullptr;
    W = KWork();
    c->kr_restart = 0;
}

void free_lowrank(pslr_ctx *c) {
    cfree(c->d_V); cfree(c->d_Vr); cfree(c->d_Vb); cfree(c->d_G); cfree(c->d_GT);
    cfree(c->d_Gf); cfree(c->d_GTf); cfree(c->d_part);
    c->d_V = nullptr; c->d_Vr = nullptr; c->d_Vb = nullptr; c->d_G = c->d_GT = nullptr; c->d_Gf = c->d_GTf = nullptr;
    c->d_part = nullptr;
    c->r = 0;
    ++c->lr_gen;
    drop_graphs(c);
    c->V.clear(); c->H.clear(); c->G.clear();
}

// Per-subdomain local structures, kept only during set-up.
struct Local {
    Csr B, E, F, C0, Cg;        // Cg columns are global interface indices
    Csr BL, BU, CL, CU;         // factors
    std::vector<uint16_t> bpiv, cpiv;
};

// The segments of subdomain i in one direction, in the order
// [E, F, Cg, B1, B2, C1, C2] (transposed: Cg left empty, inserted later),
// into its own store; k receives the kNCnt segment counts.
// Sweep levels are merged into segments no larger than the largest one-level
// segment of the precision (a full level of 3-entry records in FP64, a
// 256-row slice of a product with global columns in FP32), so merging does
// not enlarge the ring's slots.
template <class T>
constexpr int merge_budget() { return sizeof(T) == 8 ? kSegBudget : 8 * 1024; }

// The diagonal of an upper factor, row by row.
std::vector<double> upper_diag(const Csr &U) {
    std::vector<double> d(U.nr, 1.0);
    for (int r = 0; r < U.nr; ++r)
        for (int k = U.rp[r]; k < U.rp[r + 1]; ++k)
            if (U.ci[k] == r) d[r] = U.v[k];
    return d;
}

// Unit-diagonal form of the forward solves (no row pivots): with D =
// diag(1/u_rr) of the local U factor, L~ = D L D^{-1} (entries l_rk u_kk /
// u_rr) and U^ = D U (entries u_rk / u_rr, diagonal 1) give L U = D^{-1} L~ U^,
// so x = U^{-1} L^{-1} b = U^^{-1} L~^{-1} (D b): the same solve with the
// right-hand side scaled by D and no scaling multiply in either sweep.
void unit_rows(std::vector<Row> &rows, const std::vector<double> &u, bool lower) {
    for (Row &R : rows) {
        for (auto &e : R.e) e.second = lower ? e.second * u[e.first] / u[R.row] : e.second / u[R.row];
        R.diag = 1.0;
    }
}

template <class T>
void pack_subdomain(const Local &Lc, int npi, int nqi, bool transposed, int q, SegStore &S, int *k, int &levB,
                    int &levC, bool merge, bool unit = false) {
    levB = levC = 0;
    const int budget = merge ? merge_budget<T>() : 0;  // budget 0: one level per segment
    if (!transposed) {
        // unit: E's rows feed the B solves' right-hand sides, so they carry D_B
        const std::vector<double> uB = unit ? upper_diag(Lc.BU) : std::vector<double>();
        const std::vector<double> uC = unit ? upper_diag(Lc.CU) : std::vector<double>();
        std::vector<Row> er = ell_rows(Lc.E);
        if (unit)
            for (Row &R : er)
                for (auto &e : R.e) e.second /= uB[R.row];
        k[kE] = pack_rows<T, uint16_t>(S, er, false, nqi);
        k[kF] = pack_rows<T, uint16_t>(S, ell_rows(Lc.F), false, npi);
        k[kCg] = pack_rows<T, int32_t>(S, ell_rows(Lc.Cg), false, q);
        auto lb = levels(Lc.BL, true), ub = levels(Lc.BU, false);
        auto lc = levels(Lc.CL, true), uc = levels(Lc.CU, false);
        levB = (int)(lb.size() + ub.size());
        levC = (int)(lc.size() + uc.size());
        auto sweep = [&](const Csr &Tm, const std::vector<int> &lv, bool lower, const std::vector<double> &u) {
            std::vector<Row> rows = sweep_rows(Tm, lv, lower, !lower);
            if (unit) unit_rows(rows, u, lower);
            return rows;
        };
        size_t d0 = S.desc.size();
        for (auto &lv : lb) pack_rows<T, uint16_t>(S, sweep(Lc.BL, lv, true, uB), false, npi, merge);
        k[kB1] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : ub) pack_rows<T, uint16_t>(S, sweep(Lc.BU, lv, false, uB), !unit, npi, merge);
        k[kB2] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : lc) pack_rows<T, uint16_t>(S, sweep(Lc.CL, lv, true, uC), false, nqi, merge);
        k[kC1] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : uc) pack_rows<T, uint16_t>(S, sweep(Lc.CU, lv, false, uC), !unit, nqi, merge);
        k[kC2] = merge_levels(S, d0, budget);
    } else {
        // E-slot: F_i^T (interior rows <- interface cols); F-slot: E_i^T.
        k[kE] = pack_rows<T, uint16_t>(S, ell_rows(transpose(Lc.F)), false, nqi);
        k[kF] = pack_rows<T, uint16_t>(S, ell_rows(transpose(Lc.E)), false, npi);
        k[kCg] = 0;  // C_g^T rows need C_g of every subdomain: packed by pack_direction
        // B^{-T} = U^{-T} L^{-T}: sweep 1 is U^T (lower, with diagonal), sweep 2 L^T (upper)
        Csr BUt = transpose(Lc.BU), BLt = transpose(Lc.BL);
        Csr CUt = transpose(Lc.CU), CLt = transpose(Lc.CL);
        auto l1 = levels(BUt, true), l2 = levels(BLt, false);
        auto l3 = levels(CUt, true), l4 = levels(CLt, false);
        size_t d0 = S.desc.size();
        for (auto &lv : l1) pack_rows<T, uint16_t>(S, sweep_rows(BUt, lv, true, true), true, npi, merge);
        k[kB1] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : l2) pack_rows<T, uint16_t>(S, sweep_rows(BLt, lv, false, false), false, npi, merge);
        k[kB2] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : l3) pack_rows<T, uint16_t>(S, sweep_rows(CUt, lv, true, true), true, nqi, merge);
        k[kC1] = merge_levels(S, d0, budget);
        d0 = S.desc.size();
        for (auto &lv : l4) pack_rows<T, uint16_t>(S, sweep_rows(CLt, lv, false, false), false, nqi, merge);
        k[kC2] = merge_levels(S, d0, budget);
    }
}

// Every subdomain packed on its own thread into its own stores, then copied
// into one store in subdomain order.  The bytes are the main segments of
// every subdomain in turn and, in the transposed direction, the C_g^T
// segments of every subdomain after them; each subdomain's descriptors are in
// the order [E, F, Cg, B1, B2, C1, C2].  The result does not depend on the
// number of threads.
template <class T>
bool pack_direction(const std::vector<Local> &loc, const std::vector<int> &np, const std::vector<int> &nq,
                    bool transposed, int q, const std::vector<Csr> *cgT, int threads, SegStore &S,
                    std::vector<int32_t> &sub_desc, std::vector<int32_t> &cnt, int &levB, int &levC, bool merge,
                    bool unit = false) {
    const int s = (int)loc.size();
    sub_desc.assign(s, 0);
    cnt.assign((size_t)kNCnt * s, 0);
    std::vector<SegStore> part(s), pcg(transposed ? s : 0);
    std::vector<int> lb(s, 0), lc(s, 0);
    bool ok = parallel_for(s, threads, [&](int i) {
        int *k = &cnt[(size_t)kNCnt * i];
        pack_subdomain<T>(loc[i], np[i], nq[i], transposed, q, part[i], k, lb[i], lc[i], merge, unit);
        if (transposed) k[kCg] = pack_rows<T, int32_t>(pcg[i], ell_rows((*cgT)[i]), false, q);
    });
    if (!ok) return false;
    std::vector<int64_t> boff(s), coff(s);
    int64_t total = 0;
    size_t nd = 0;
    for (int i = 0; i < s; ++i) {
        boff[i] = total;
        total += (int64_t)part[i].bytes.size();
        sub_desc[i] = (int32_t)nd;
        nd += part[i].desc.size() + (transposed ? pcg[i].desc.size() : 0);
        S.max_bytes = std::max(S.max_bytes, part[i].max_bytes);
        levB = std::max(levB, lb[i]);
        levC = std::max(levC, lc[i]);
    }
    for (int i = 0; i < (int)pcg.size(); ++i) {
        coff[i] = total;
        total += (int64_t)pcg[i].bytes.size();
        S.max_bytes = std::max(S.max_bytes, pcg[i].max_bytes);
    }
    S.bytes.resize((size_t)total);
    S.desc.resize(nd);
    return parallel_for(s, threads, [&](int i) {
        SegStore &P = part[i];
        if (!P.bytes.empty()) std::memcpy(S.bytes.data() + boff[i], P.bytes.data(), P.bytes.size());
        SegDesc *d = S.desc.data() + sub_desc[i];
        const int *k = &cnt[(size_t)kNCnt * i];
        const size_t head = transposed ? (size_t)(k[kE] + k[kF]) : P.desc.size();
        auto put = [&](SegDesc x, int64_t base) {
            x.off += base;
            *d++ = x;
        };
        for (size_t t = 0; t < head; ++t) put(P.desc[t], boff[i]);
        if (transposed) {
            SegStore &Q = pcg[i];
            if (!Q.bytes.empty()) std::memcpy(S.bytes.data() + coff[i], Q.bytes.data(), Q.bytes.size());
            for (const SegDesc &x : Q.desc) put(x, coff[i]);
            Q = SegStore();
        }
        for (size_t t = head; t < P.desc.size(); ++t) put(P.desc[t], boff[i]);
        P = SegStore();
    });
}

}  // namespace

// Host-side check of a packed layout (pslr_plan): it decodes every segment
// the kernels will read and counts violations of what they rely on.
//  - every header is consistent (rows <= kSegMaxRows, padding, encoding,
//    byte size) and every row and column index is in range for its block
//    (columns may name the zero slot: an unused entry);
//  - an E, F or C_g product writes each output row at most once (its warps
//    run through the segments without a barrier);
//  - a triangular sweep writes every row of its block exactly once, and each
//    row reads only rows written at an earlier barrier step of the same sweep
//    (one block of a segment is one barrier step), so no two threads race;
//  - a segment's blocks fill it exactly, and only sweeps chain blocks.
template <class T>
static int64_t check_layout(const pslr_ctx *c, const SegStore &S, const std::vector<int32_t> &sub_desc,
                            const std::vector<int32_t> &cnt, std::string *first) {
    int64_t bad = 0;
    auto note = [&](const char *what, int i, int cat) {
        if (bad++ == 0 && first) {
            char buf[160];
            snprintf(buf, sizeof buf, "layout check: %s (subdomain %d, segment kind %d)", what, i, cat);
            *first = buf;
        }
    };
    std::vector<int> step;
    for (int i = 0; i < c->s; ++i) {
        const int np = c->ioff[i + 1] - c->ioff[i], nq = c->goff[i + 1] - c->goff[i];
        int d = sub_desc[i];
        for (int cat = 0; cat < kNCnt; ++cat) {
            const bool sweep = cat >= kB1;
            const int nrows = (cat == kE || cat == kB1 || cat == kB2) ? np : nq;
            const int ncols = cat == kE ? nq : cat == kF ? np : cat == kCg ? c->q : nrows;  // also the zero slot
            step.assign((size_t)nrows, -1);
            const int nseg = cnt[(size_t)kNCnt * i + cat];
            int stepno = 0;  // barrier steps so far: one per block
            for (int t = 0; t < nseg; ++t, ++d) {
                const SegDesc &sd = S.desc[d];
                if (sd.off < 0 || sd.off + sd.bytes > (int64_t)S.bytes.size() || sd.bytes < (int)sizeof(SegHdr)) {
                    note("segment outside the store", i, cat);
                    continue;
                }
                int64_t boff = 0;
                for (;; ++stepno) {
                if (boff + (int64_t)sizeof(SegHdr) > sd.bytes) {
                    note("a segment's blocks run past its end", i, cat);
                    break;
                }
                const char *base = S.bytes.data() + sd.off + boff;
                SegHdr h;
                std::memcpy(&h, base, sizeof h);
                const bool global = (h.flags & kSegGlobalCols) != 0, diag = (h.flags & kSegDiag) != 0;
                const bool more = (h.flags & kSegMore) != 0;
                const int n = h.n, pn = h.np, fmt = h.fmt;
                const int w = fmt == kTile ? h.w : fmt;
                const int64_t raw = global ? seg_bytes<T, int32_t>(n, w, diag) : seg_bytes<T, uint16_t>(n, w, diag);
                // levels of merged sweep segments are padded to 128 bytes
                const int64_t want = sweep && (int64_t)h.bytes == align_up((int)raw, 128) ? align_up((int)raw, 128) : raw;
                if (n < 1 || n > kSegMaxRows || pn != seg_npad(n) || global != (cat == kCg) ||
                    (fmt != kTile && fmt != kRec3 && fmt != kRec7) || seg_fmt_for(w) != fmt ||
                    want != (int64_t)h.bytes || boff + want > sd.bytes || (more && !sweep) ||
                    (!more && boff + want != sd.bytes)) {
                    note("inconsistent segment header", i, cat);
                    break;
                }
                const int tstep = sweep ? stepno : t;
                auto idx = [&](size_t k) -> int {
                    if (global) {
                        int32_t x;
                        std::memcpy(&x, base + sizeof(SegHdr) + 4 * k, 4);
                        return x;
                    }
                    uint16_t x;
                    std::memcpy(&x, base + sizeof(SegHdr) + 2 * k, 2);
                    return x;
                };
                const size_t isz = global ? 4 : 2;
                std::vector<std::pair<int, int>> writes;  // (row, step) applied after the block
                for (int j = 0; j < n; ++j) {
                    int row;
                    if (fmt != kTile) {
                        row = idx((size_t)j * (w + 1));
                    } else {
                        const size_t roff = sizeof(SegHdr) + (size_t)pn * w * sizeof(T) + (diag ? pn * sizeof(T) : 0) +
                                            (size_t)pn * w * isz;
                        uint16_t r16;
                        std::memcpy(&r16, base + roff + 2 * (size_t)j, 2);
                        row = r16;
                    }
                    if (row < 0 || row >= nrows) {
                        note("row out of range", i, cat);
                        continue;
                    }
                    for (int k = 0; k < w; ++k) {
                        int col;
                        if (fmt != kTile) {
                            col = idx((size_t)j * (w + 1) + 1 + k);
                        } else {
                            const size_t coff = sizeof(SegHdr) + (size_t)pn * w * sizeof(T) + (diag ? pn * sizeof(T) : 0);
                            if (global) {
                                int32_t x;
                                std::memcpy(&x, base + coff + 4 * ((size_t)k * pn + j), 4);
                                col = x;
                            } else {
                                uint16_t x;
                                std::memcpy(&x, base + coff + 2 * ((size_t)k * pn + j), 2);
                                col = x;
                            }
                        }
                        if (col < 0 || col > ncols) {
                            note("column out of range", i, cat);
                        } else if (sweep && col < ncols && (step[col] < 0 || step[col] >= tstep)) {
                            note("a sweep row reads a row not written at an earlier step", i, cat);
                        }
                    }
                    writes.push_back({row, tstep});
                }
                for (auto &wr : writes) {
                    if (step[wr.first] >= 0) note(sweep ? "a sweep writes a row twice" : "a product writes a row twice", i, cat);
                    step[wr.first] = wr.second;
                }
                if (!more) {
                    ++stepno;
                    break;
                }
                boff += want;
                }
            }
            if (sweep)
                for (int r = 0; r < nrows; ++r)
                    if (step[r] < 0) {
                        note("a sweep leaves a row unwritten", i, cat);
                        break;
                    }
        }
    }
    return bad;
}

template <class T>
static pslr_status finish_opset(pslr_ctx *c, OpSetHost &o, SegStore &S, const std::vector<int32_t> &sub_desc,
                                const std::vector<int32_t> &cnt, bool fp32, bool plan_only) {
    o.slot_bytes = align_up(std::max(S.max_bytes, 128), 128);
    o.seg_total = (int64_t)S.bytes.size();
    for (int i = 0; i < c->s; ++i) {
        int d = sub_desc[i];
        for (int k = 0; k < kNCnt; ++k)
            for (int t = 0; t < cnt[(size_t)kNCnt * i + k]; ++t) o.cat_bytes[k] += S.desc[d++].bytes;
    }
    o.hdesc = S.desc;
    o.hsub = sub_desc;
    o.hcnt = cnt;
    if (plan_only) {
        std::string first;
        c->layout_errors += check_layout<T>(c, S, sub_desc, cnt, c->layout_errors ? nullptr : &first);
        if (!first.empty()) fprintf(stderr, "pslr_plan: %s\n", first.c_str());
        uint64_t h = c->layout_hash ? c->layout_hash : 0xcbf29ce484222325ull;
        h = fnv1a(h, S.bytes.data(), S.bytes.size());
        for (const SegDesc &d : S.desc) {  // field by field: the struct has padding
            h = fnv1a(h, &d.off, sizeof(d.off));
            h = fnv1a(h, &d.bytes, sizeof(d.bytes));
        }
        h = fnv1a(h, sub_desc.data(), sub_desc.size() * sizeof(int32_t));
        c->layout_hash = fnv1a(h, cnt.data(), cnt.size() * sizeof(int32_t));
    }
    if (S.bytes.empty()) S.bytes.resize(16, 0);
    const bool piv = c->factor == 1;
    int optin = 227 * 1024;  // sm_100-class opt-in limit; queried from the device when there is one
    if (!plan_only) {
        CK(upload(&o.seg, S.bytes));
        CK(upload(&o.cnt, cnt));
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    }
    // ring depth: as many slots as fit next to the vectors, 2 .. kMaxRing; checked
    // here for the largest rank, so that every later low-rank term fits (the
    // launch shape itself is chosen by plan_launch for the current rank)
    const int avail = optin - 1024 - smem_fixed(c->max_p, c->max_q, fp32 ? 4 : 8, piv, kMaxRank, true);
    o.ring = std::min(kMaxRing, avail / o.slot_bytes);
    if (o.ring < 2)
        return fail(c, PSLR_ERR_TOO_LARGE,
                    "a subdomain needs more shared memory than one CTA has (%d interior, %d interface "
                    "unknowns): use more subdomains", c->max_p, c->max_q);
    o.smem = smem_layout(o.slot_bytes, o.ring, c->max_p, c->max_q, fp32 ? 4 : 8, piv, kMaxRank, true).total;
    o.grid = 0;
    return PSLR_OK;
}

// ------------------------------------------------------------------- C ABI

extern "C" {

const char *pslr_status_string(pslr_status s) {
    switch (s) {
    case PSLR_OK: return "ok";
    case PSLR_ERR_ARG: return "invalid argument";
    case PSLR_ERR_CUDA: return "CUDA error";
    case PSLR_ERR_ZERO_PIVOT: return "zero pivot in a local factorization";
    case PSLR_ERR_BREAKDOWN: return "Arnoldi breakdown (rank truncated)";
    case PSLR_ERR_SINGULAR_IMH: return "I - H is singular";
    case PSLR_ERR_NOT_CONVERGED: return "FGMRES did not converge";
    case PSLR_ERR_NAN: return "NaN or Inf";
    case PSLR_ERR_TIMEOUT: return "device-side wait timed out";
    case PSLR_ERR_STATE: return "call out of order";
    case PSLR_ERR_TOO_LARGE: return "subdomain too large";
    }
    return "unknown status";
}

const char *pslr_last_error(const pslr_ctx *c) { return c ? c->err.c_str() : "null context"; }

void pslr_destroy(pslr_ctx *c) {
    if (!c) return;
    for (auto &d : c->ops)
        for (auto &o : d) free_opset(o);
    free_opset(c->ops_unit);
    cfree(c->d_dB);
    cfree(c->d_dC);
    free_krylov(c);
    free_lowrank(c);
    if (c->kcap) cudaStreamDestroy(c->kcap);
    if (c->h_err) cudaFreeHost(c->h_err);
    for (void *p : {(void *)c->d_perm, (void *)c->d_ioff, (void *)c->d_goff, (void *)c->d_bpiv,
                    (void *)c->d_cpiv, (void *)c->d_rp, (void *)c->d_ci, (void *)c->d_rpT, (void *)c->d_ciT,
                    (void *)c->d_av, (void *)c->d_avT, (void *)c->d_wbuf, (void *)c->d_acc, (void *)c->d_bar,
                    (void *)c->d_err, (void *)c->d_eab, c->d_io_b, c->d_io_z})
        cfree(p);
    delete c;
}

}  // extern "C"

static pslr_status prebuild_streams(pslr_ctx *c);

// Launch shape of the persistent kernels for the current rank: per precision
// the ring depth, dynamic shared memory, cooperative grid and CTAs per SM
// (both directions share one shape).  One CTA per SM takes the deepest ring
// that fits; when the subdomains outnumber the resident CTAs and two CTAs fit
// an SM with at least kMinDualRing slots each, the two-CTAs-per-SM instances
// run instead, so that no CTA sweeps two subdomains in sequence.  The
// low-rank scratch is sized for the current rank (red_stride), so the shape is
// planned again whenever the low-rank term changes; segment streams built for
// another grid are dropped.
static pslr_status plan_launch(pslr_ctx *c) {
    int dev = 0, optin = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int rs = red_stride(c->r);
    const bool piv = c->factor == 1;
    for (int prec = 0; prec < 2; ++prec) {
        const int ts = prec == 0 ? 8 : 4;
        // the operator sets launched with this precision's kernels share one shape
        std::vector<OpSetHost *> sets = {&c->ops[0][prec], &c->ops[1][prec]};
        if (prec == 0 && c->has_unit) sets.push_back(&c->ops_unit);
        const int ns = (int)sets.size();
        auto shape = [&](int budget, int *ring, int *smem) {
            const int avail = budget - 1024 - smem_fixed(c->max_p, c->max_q, ts, piv, rs, true);
            *smem = 0;
            for (int d = 0; d < ns; ++d) {
                ring[d] = std::min(kMaxRing, avail / sets[d]->slot_bytes);
                *smem = std::max(*smem, smem_layout(sets[d]->slot_bytes, ring[d], c->max_p, c->max_q, ts, piv, rs,
                                                    true).total);
            }
        };
        auto min_ring = [&](const int *ring) {
            int m = ring[0];
            for (int d = 1; d < ns; ++d) m = std::min(m, ring[d]);
            return m;
        };
        int ring[3], smem = 0;
        shape(optin, ring, &smem);
        if (min_ring(ring) < 2)
            return fail(c, PSLR_ERR_TOO_LARGE, "a subdomain needs more shared memory than one CTA has");
        const bool merged = c->ops[0][prec].merged;  // the same for every set of the precision
        int cap = max_coresident_apply(smem, prec == 1, false, merged);
        if (cap <= 0) return fail(c, PSLR_ERR_CUDA, "persistent kernel cannot be made resident");
        bool dual = false;
        if (c->s > cap) {
            int ring2[3], smem2 = 0;
            shape(per_sm / 2, ring2, &smem2);
            if (min_ring(ring2) >= kMinDualRing) {
                const int cap2 = max_coresident_apply(smem2, prec == 1, true, merged);
                if (cap2 > cap) {
                    dual = true;
                    cap = cap2;
                    smem = smem2;
                    for (int d = 0; d < ns; ++d) ring[d] = ring2[d];
                }
            }
        }
        const int grid = std::min(cap, c->s);
        for (int d = 0; d < ns; ++d) {
            OpSetHost &o = *sets[d];
            if (o.grid != grid) {  // streams partition the subdomains over the grid
                for (auto &kv : o.streams) {
                    cfree(kv.second.ent);
                    cfree(kv.second.off);
                }
                o.streams.clear();
            }
            o.ring = ring[d];
            o.smem = smem;
            o.grid = grid;
            o.dual = dual;
        }
    }
    c->rs = rs;
    drop_graphs(c);
    return PSLR_OK;
}

// Everything pslr_setup does; with plan_only the device is never touched (no
// uploads, no allocations), which pslr_plan uses.
static pslr_status setup_impl(pslr_ctx *c, int32_t n, const int32_t *rowptr, const int32_t *colind,
                              const double *val, const pslr_opts *opts, bool plan_only) {
    auto bail = [](pslr_status st) { return st; };
    c->n = n;
    c->factor = opts->factor;
    c->seed = opts->seed;
    if (opts->factor < 0 || opts->factor > 2) return bail(fail(c, PSLR_ERR_ARG, "factor must be 0, 1 or 2"));
    if (opts->factor == 2 && !(opts->drop_tol >= 0.0 && std::isfinite(opts->drop_tol)))
        return bail(fail(c, PSLR_ERR_ARG, "ILUT needs a finite drop tolerance >= 0"));
    c->drop_tol = opts->drop_tol;
    if (opts->merge_levels < 0 || opts->merge_levels > 2)
        return bail(fail(c, PSLR_ERR_ARG, "merge_levels must be 0, 1 or 2"));
    c->merge_levels = opts->merge_levels;
    if (opts->device_factor < 0 || opts->device_factor > 1)
        return bail(fail(c, PSLR_ERR_ARG, "device_factor must be 0 or 1"));
    if (opts->device_factor == 1 && opts->factor != 0)
        return bail(fail(c, PSLR_ERR_ARG, "device_factor needs ILU(0) local factors (factor 0)"));
    c->device_factor = plan_only ? 0 : opts->device_factor;
    if (opts->setup_threads < 0) return bail(fail(c, PSLR_ERR_ARG, "setup_threads must be >= 0"));
    if (opts->setup_threads > 0) {
        c->threads = opts->setup_threads;
    } else {
        const unsigned hw = std::thread::hardware_concurrency();
        c->threads = (int)std::min(64u, std::max(1u, hw));
    }
    const int threads = c->threads;
    // --- validate CSR: monotone row pointers, columns in range and ascending, diagonal present
    if (rowptr[0] != 0) return bail(fail(c, PSLR_ERR_ARG, "rowptr[0] != 0"));
    for (int i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return bail(fail(c, PSLR_ERR_ARG, "rowptr not monotone at %d", i));
        bool diag = false;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int j = colind[k];
            if (j < 0 || j >= n) return bail(fail(c, PSLR_ERR_ARG, "column %d out of range in row %d", j, i));
            if (k > rowptr[i] && colind[k - 1] >= j)
                return bail(fail(c, PSLR_ERR_ARG, "columns not strictly ascending in row %d", i));
            if (!std::isfinite(val[k])) return bail(fail(c, PSLR_ERR_ARG, "non-finite value in row %d", i));
            diag |= (j == i);
        }
        if (!diag) return bail(fail(c, PSLR_ERR_ZERO_PIVOT, "row %d has no diagonal entry", i));
    }
    const int64_t nnz = rowptr[n];
    c->nnz_A = nnz;
    c->h_rp.assign(rowptr, rowptr + n + 1);
    c->h_ci.assign(colind, colind + nnz);
    c->h_av.assign(val, val + nnz);

    // --- Section 2: partition and reordering
    c->part.resize(n);
    if (opts->part) {
        int mx = -1;
        for (int v = 0; v < n; ++v) {
            if (opts->part[v] < 0) return bail(fail(c, PSLR_ERR_ARG, "negative part id"));
            c->part[v] = opts->part[v];
            mx = std::max(mx, (int)opts->part[v]);
        }
        c->s = mx + 1;
    } else if (opts->dims[0] == 0 && opts->dims[1] == 0 && opts->dims[2] == 0 && opts->nparts > 0) {
        if (opts->nparts > n) return bail(fail(c, PSLR_ERR_ARG, "nparts exceeds n"));
        if (!pslr_part::graph_partition(n, rowptr, colind, opts->nparts, c->part.data(), threads))
            return bail(fail(c, PSLR_ERR_ARG, "graph partition failed (out of host memory)"));
        c->s = opts->nparts;
    } else {
        const int64_t Nx = opts->dims[0], Ny = opts->dims[1], Nz = opts->dims[2];
        const int Px = opts->splits[0], Py = opts->splits[1], Pz = opts->splits[2];
        if (Nx <= 0 || Ny <= 0 || Nz <= 0 || Nx * Ny * Nz != n)
            return bail(fail(c, PSLR_ERR_ARG, "dims do not multiply to n"));
        if (Px < 1 || Py < 1 || Pz < 1 || Px > Nx || Py > Ny || Pz > Nz)
            return bail(fail(c, PSLR_ERR_ARG, "splits out of range"));
        for (int64_t v = 0; v < n; ++v) {
            int64_t i = v % Nx, j = (v / Nx) % Ny, k = v / (Nx * Ny);
            c->part[v] = (int32_t)((i * Px) / Nx + Px * ((j * Py) / Ny + Py * ((k * Pz) / Nz)));
        }
        c->s = Px * Py * Pz;
    }
    const int s = c->s;
    c->iface.assign(n, 0);
    for (int v = 0; v < n; ++v)
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            int w = colind[k];
            if (w != v && c->part[w] != c->part[v]) c->iface[v] = c->iface[w] = 1;
        }
    // counting sort by (interface?, part, index): stable in the original index
    std::vector<int64_t> cntI(s + 1, 0), cntG(s + 1, 0);
    for (int v = 0; v < n; ++v) (c->iface[v] ? cntG : cntI)[c->part[v] + 1]++;
    for (int i = 0; i < s; ++i) {
        cntI[i + 1] += cntI[i];
        cntG[i + 1] += cntG[i];
    }
    c->p = (int)cntI[s];
    c->q = (int)cntG[s];
    c->ioff.assign(cntI.begin(), cntI.end());
    c->goff.assign(cntG.begin(), cntG.end());
    c->perm.assign(n, 0);
    std::vector<int32_t> loc(n), posI(c->ioff.begin(), c->ioff.end() - 1), posG(c->goff.begin(), c->goff.end() - 1);
    for (int v = 0; v < n; ++v) {
        int i = c->part[v];
        if (c->iface[v]) {
            loc[v] = posG[i] - c->goff[i];
            c->perm[c->p + posG[i]++] = v;
        } else {
            loc[v] = posI[i] - c->ioff[i];
            c->perm[posI[i]++] = v;
        }
    }
    std::vector<int> np(s), nq(s);
    for (int i = 0; i < s; ++i) {
        np[i] = c->ioff[i + 1] - c->ioff[i];
        nq[i] = c->goff[i + 1] - c->goff[i];
        c->max_p = std::max(c->max_p, np[i]);
        c->max_q = std::max(c->max_q, nq[i]);
    }
    if (c->max_p >= 65535 || c->max_q >= 65535)
        return bail(fail(c, PSLR_ERR_TOO_LARGE, "a subdomain has more than 65534 interior or interface unknowns"));

    // --- Eq. 2.1 / Eq. 3.1: local blocks (rows visited in the reordered order)
    std::vector<Local> L(s);
    bool blocks_ok = parallel_for(s, threads, [&](int i) {
        Local &Lc = L[i];
        for (Csr *M : {&Lc.B, &Lc.E}) { M->nr = np[i]; M->rp.assign(1, 0); }
        for (Csr *M : {&Lc.F, &Lc.C0, &Lc.Cg}) { M->nr = nq[i]; M->rp.assign(1, 0); }
        Lc.B.nc = np[i]; Lc.E.nc = nq[i]; Lc.F.nc = np[i]; Lc.C0.nc = nq[i]; Lc.Cg.nc = c->q;
        for (int t = 0; t < np[i]; ++t) {
            int v = c->perm[c->ioff[i] + t];
            for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                int w = colind[k];
                Csr &M = c->iface[w] ? Lc.E : Lc.B;
                M.ci.push_back(loc[w]);
                M.v.push_back(val[k]);
            }
            Lc.B.rp.push_back((int32_t)Lc.B.ci.size());
            Lc.E.rp.push_back((int32_t)Lc.E.ci.size());
        }
        for (int t = 0; t < nq[i]; ++t) {
            int v = c->perm[c->p + c->goff[i] + t];
            std::vector<std::pair<int32_t, double>> cg;
            for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                int w = colind[k];
                if (!c->iface[w]) {
                    Lc.F.ci.push_back(loc[w]);
                    Lc.F.v.push_back(val[k]);
                } else if (c->part[w] == i) {
                    Lc.C0.ci.push_back(loc[w]);
                    Lc.C0.v.push_back(val[k]);
                } else {
                    cg.push_back({c->goff[c->part[w]] + loc[w], val[k]});
                }
            }
            std::sort(cg.begin(), cg.end());
            for (auto &e : cg) {
                Lc.Cg.ci.push_back(e.first);
                Lc.Cg.v.push_back(e.second);
            }
            Lc.F.rp.push_back((int32_t)Lc.F.ci.size());
            Lc.C0.rp.push_back((int32_t)Lc.C0.ci.size());
            Lc.Cg.rp.push_back((int32_t)Lc.Cg.ci.size());
        }
    });
    if (!blocks_ok) return bail(fail(c, PSLR_ERR_ARG, "host set-up failed while extracting the blocks (out of memory?)"));

    // --- Algorithm 1, steps 2-5: local factors
    // With device_factor, all B_i and C_i are factored at once on the GPU as
    // one block-diagonal matrix (B_0 .. B_{s-1}, then C_0 .. C_{s-1}); dev_v
    // receives the factored values in that order.
    std::vector<double> dev_v;
    // offsets of each block's rows and stored entries in that matrix
    std::vector<int32_t> bptr(2 * s + 1, 0);
    std::vector<int64_t> dev_off(2 * s + 1, 0);
    for (int b = 0; b < 2 * s; ++b) {
        const Csr &M = b < s ? L[b].B : L[b - s].C0;
        bptr[b + 1] = bptr[b] + M.nr;
        dev_off[b + 1] = dev_off[b] + (int64_t)M.v.size();
    }
    if (c->device_factor) {
        if (dev_off[2 * s] > INT32_MAX)
            return bail(fail(c, PSLR_ERR_TOO_LARGE, "device factor: more than 2^31 stored entries in B and C0"));
        std::vector<int32_t> rp(bptr[2 * s] + 1, 0), ci(dev_off[2 * s]);
        dev_v.resize(dev_off[2 * s]);
        parallel_for(2 * s, threads, [&](int b) {
            const Csr &M = b < s ? L[b].B : L[b - s].C0;
            const int r0 = bptr[b];
            const int64_t e0 = dev_off[b];
            for (int r = 0; r < M.nr; ++r) rp[r0 + r + 1] = (int32_t)(e0 + M.rp[r + 1]);
            for (size_t k = 0; k < M.v.size(); ++k) {
                ci[e0 + k] = r0 + M.ci[k];
                dev_v[e0 + k] = M.v[k];
            }
        });
        double *d_v = nullptr;
        cudaError_t e = cudaMalloc(&d_v, std::max<size_t>(1, dev_v.size()) * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(d_v, dev_v.data(), dev_v.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d_v);
            return bail(fail(c, PSLR_ERR_CUDA, "device factor: %s", cudaGetErrorString(e)));
        }
        int bad = -1;
        std::string why;
        const pslr_status fst = ilu0_device_blocks(bptr.back(), 2 * s, bptr.data(), rp.data(), ci.data(), d_v,
                                                   nullptr, &c->factor_ms, &bad, why);
        if (fst == PSLR_OK)
            e = cudaMemcpy(dev_v.data(), d_v, dev_v.size() * sizeof(double), cudaMemcpyDeviceToHost);
        cudaFree(d_v);
        if (fst == PSLR_ERR_ZERO_PIVOT) {
            // the block of the first failing row: B_i for rows below p, else C_i
            const int blk = (int)(std::upper_bound(bptr.begin(), bptr.end(), bad) - bptr.begin()) - 1;
            return bail(fail(c, PSLR_ERR_ZERO_PIVOT, "ILU(0) met a zero pivot in subdomain %d", blk % s));
        }
        if (fst != PSLR_OK) return bail(fail(c, fst, "device factor: %s", why.c_str()));
        if (e != cudaSuccess) return bail(fail(c, PSLR_ERR_CUDA, "device factor: %s", cudaGetErrorString(e)));
    }
    std::vector<uint16_t> bpiv, cpiv;
    if (c->factor == 1) {
        bpiv.resize(c->p);
        cpiv.resize(c->q);
    }
    // every subdomain on its own thread; the first failing subdomain (lowest
    // index) is reported, as a serial loop would
    enum { kFacOk = 0, kFacZeroPivot, kFacTooLarge };
    std::vector<int> fac_st(s, kFacOk);
    std::vector<int64_t> fac_nnz(s, 0), fac_b(s, 0);
    bool fac_ok = parallel_for(s, threads, [&](int i) {
        Local &Lc = L[i];
        Csr fb, fc;
        if (c->factor == 0 && c->device_factor) {
            fb = Lc.B;
            fc = Lc.C0;
            std::copy(dev_v.begin() + dev_off[i], dev_v.begin() + dev_off[i + 1], fb.v.begin());
            std::copy(dev_v.begin() + dev_off[s + i], dev_v.begin() + dev_off[s + i + 1], fc.v.begin());
        } else if (c->factor == 0) {
            fb = Lc.B;
            fc = Lc.C0;
            if (!ilu0_inplace(fb) || !ilu0_inplace(fc)) {
                fac_st[i] = kFacZeroPivot;
                return;
            }
        } else if (c->factor == 2) {
            if (!ilut(Lc.B, c->drop_tol, fb) || !ilut(Lc.C0, c->drop_tol, fc)) {
                fac_st[i] = kFacZeroPivot;
                return;
            }
        } else {
            if (np[i] > 4096 || nq[i] > 4096) {
                fac_st[i] = kFacTooLarge;
                return;
            }
            if (!dense_lu(Lc.B, fb, Lc.bpiv) || !dense_lu(Lc.C0, fc, Lc.cpiv)) {
                fac_st[i] = kFacZeroPivot;
                return;
            }
            std::copy(Lc.bpiv.begin(), Lc.bpiv.end(), bpiv.begin() + c->ioff[i]);
            std::copy(Lc.cpiv.begin(), Lc.cpiv.end(), cpiv.begin() + c->goff[i]);
        }
        fac_nnz[i] = (int64_t)fb.ci.size() + (int64_t)fc.ci.size();
        fac_b[i] = (int64_t)fb.ci.size();
        split_lu(fb, Lc.BL, Lc.BU);
        split_lu(fc, Lc.CL, Lc.CU);
    });
    if (!fac_ok) return bail(fail(c, PSLR_ERR_ARG, "host set-up failed while factoring (out of memory?)"));
    for (int i = 0; i < s; ++i) {
        if (fac_st[i] == kFacTooLarge)
            return bail(fail(c, PSLR_ERR_TOO_LARGE, "exact local LU is limited to blocks of 4096 rows"));
        if (fac_st[i] == kFacZeroPivot) {
            const char *what = c->factor == 0 ? "ILU(0) met a zero pivot" : c->factor == 2 ? "ILUT met a zero pivot"
                                                                                             : "singular local block";
            return bail(fail(c, PSLR_ERR_ZERO_PIVOT, "%s in subdomain %d", what, i));
        }
        c->nnz_ilu += fac_nnz[i];
        c->nnz_blk[0] += fac_b[i];
        c->nnz_blk[1] += fac_nnz[i] - fac_b[i];
        c->nnz_blk[2] += (int64_t)L[i].E.ci.size();
        c->nnz_blk[3] += (int64_t)L[i].F.ci.size();
        c->nnz_blk[4] += (int64_t)L[i].Cg.ci.size();
    }

    // --- device layout: both directions, both precisions
    std::vector<Csr> cgT(s);
    {
        // rows of C_g^T owned by subdomain i: column l of C_g for l in its interface range
        std::vector<std::vector<std::pair<int32_t, double>>> colsT(c->q);
        for (int i = 0; i < s; ++i)
            for (int t = 0; t < nq[i]; ++t)
                for (int k = L[i].Cg.rp[t]; k < L[i].Cg.rp[t + 1]; ++k)
                    colsT[L[i].Cg.ci[k]].push_back({c->goff[i] + t, L[i].Cg.v[k]});
        for (int i = 0; i < s; ++i) {
            Csr &M = cgT[i];
            M.nr = nq[i];
            M.nc = c->q;
            M.rp.assign(1, 0);
            for (int t = 0; t < nq[i]; ++t) {
                auto &v = colsT[c->goff[i] + t];
                std::sort(v.begin(), v.end());
                for (auto &e : v) {
                    M.ci.push_back(e.first);
                    M.v.push_back(e.second);
                }
                M.rp.push_back((int32_t)M.ci.size());
            }
        }
    }
    // Sweep levels are merged into multi-level segments only where the ring
    // will be shallow: with more subdomains than SMs the kernels run two CTAs
    // per SM, and if that leaves room for fewer than kMergeBelowSlots segments
    // of kSegBudget bytes, one bulk copy per level cannot keep ahead of the
    // sweeps (128^3 FP64: 1025 -> 947 us merged).  With a deep ring one level
    // per segment is faster (the per-level bookkeeping of merged segments
    // costs ~8% at 64^3).  Without a device (pslr_plan) the GB300's counts
    // stand in.
    bool merge[2] = {false, false};
    {
        int nsm = 152, per_sm = 233472;
        if (!plan_only) {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        }
        for (int prec = 0; prec < 2; ++prec) {
            const int ts = prec == 0 ? 8 : 4;
            const int avail = per_sm / 2 - 1024 - smem_fixed(c->max_p, c->max_q, ts, c->factor == 1, red_stride(0), true);
            merge[prec] = c->merge_levels == 2 ||
                          (c->merge_levels == 0 && c->s > nsm && avail < kMergeBelowSlots * kSegBudget);
        }
    }
    for (int dir = 0; dir < 2; ++dir)
        for (int prec = 0; prec < 2; ++prec) {
            SegStore S;
            std::vector<int32_t> sub_desc, cnt;
            int lb = 0, lc = 0;
            pslr_status st;
            bool ok;
            c->ops[dir][prec].merged = merge[prec];
            if (prec == 0) {
                ok = pack_direction<double>(L, np, nq, dir == 1, c->q, &cgT, threads, S, sub_desc, cnt, lb, lc,
                                            merge[0]);
                st = ok ? finish_opset<double>(c, c->ops[dir][prec], S, sub_desc, cnt, false, plan_only) : PSLR_OK;
            } else {
                ok = pack_direction<float>(L, np, nq, dir == 1, c->q, &cgT, threads, S, sub_desc, cnt, lb, lc,
                                           merge[1]);
                st = ok ? finish_opset<float>(c, c->ops[dir][prec], S, sub_desc, cnt, true, plan_only) : PSLR_OK;
            }
            if (!ok) return bail(fail(c, PSLR_ERR_ARG, "host set-up failed while packing (out of memory?)"));
            if (st != PSLR_OK) return bail(st);
            if (dir == 0 && prec == 0) {
                c->levels_B = lb;
                c->levels_C = lc;
            }
        }
    if (c->factor != 1) {  // the unit-diagonal forward FP64 set (no row pivots to respect)
        SegStore S;
        std::vector<int32_t> sub_desc, cnt;
        int lb = 0, lc = 0;
        c->ops_unit.merged = merge[0];
        const bool ok = pack_direction<double>(L, np, nq, false, c->q, &cgT, threads, S, sub_desc, cnt, lb, lc,
                                               merge[0], true);
        if (!ok) return bail(fail(c, PSLR_ERR_ARG, "host set-up failed while packing (out of memory?)"));
        pslr_status st = finish_opset<double>(c, c->ops_unit, S, sub_desc, cnt, false, plan_only);
        if (st != PSLR_OK) return bail(st);
        c->h_dB.assign(c->p, 1.0);
        c->h_dC.assign(c->q, 1.0);
        for (int i = 0; i < c->s; ++i) {
            const std::vector<double> uB = upper_diag(L[i].BU), uC = upper_diag(L[i].CU);
            for (int r = 0; r < (int)uB.size(); ++r) c->h_dB[c->ioff[i] + r] = 1.0 / uB[r];
            for (int r = 0; r < (int)uC.size(); ++r) c->h_dC[c->goff[i] + r] = 1.0 / uC[r];
        }
        c->has_unit = true;
    }
    if (plan_only) return PSLR_OK;
    {
        pslr_status ps = plan_launch(c);
        if (ps != PSLR_OK) return bail(ps);
    }
    CK(upload(&c->d_perm, c->perm));
    CK(upload(&c->d_ioff, c->ioff));
    CK(upload(&c->d_goff, c->goff));
    if (c->factor == 1) {
        CK(upload(&c->d_bpiv, bpiv));
        CK(upload(&c->d_cpiv, cpiv));
    }
    if (c->has_unit) {
        CK(upload(&c->d_dB, c->h_dB));
        CK(upload(&c->d_dC, c->h_dC));
    }
    CK(upload(&c->d_rp, c->h_rp));
    CK(upload(&c->d_ci, c->h_ci));
    CK(upload(&c->d_av, c->h_av));
    {
        Csr A;
        A.nr = A.nc = n;
        A.rp = c->h_rp;
        A.ci = c->h_ci;
        A.v = c->h_av;
        Csr At = transpose(A);
        CK(upload(&c->d_rpT, At.rp));
        CK(upload(&c->d_ciT, At.ci));
        CK(upload(&c->d_avT, At.v));
    }
    CK(cudaMalloc(&c->d_wbuf, sizeof(double) * 2 * (c->q + 1)));
    CK(cudaMemset(c->d_wbuf, 0, sizeof(double) * 2 * (c->q + 1)));
    CK(cudaMalloc(&c->d_acc, sizeof(double) * (c->q + 1)));
    CK(cudaMalloc(&c->d_eab, sizeof(double) * 2 * (c->q + 1)));
    CK(cudaMalloc(&c->d_bar, 2 * sizeof(unsigned)));
    CK(cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned)));
    CK(cudaMalloc(&c->d_err, sizeof(int)));
    CK(cudaMemset(c->d_err, 0, sizeof(int)));
    CK(cudaDeviceSynchronize());
    return prebuild_streams(c);
}

extern "C" {

pslr_status pslr_setup(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
                       const pslr_opts *opts, void *stream, pslr_ctx **out) {
    TraceRange trace("pslr_setup");
    if (!out) return PSLR_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || !rowptr || !colind || !val || !opts) return PSLR_ERR_ARG;
    (void)stream;
    pslr_ctx *c = new pslr_ctx();
    pslr_status st = setup_impl(c, n, rowptr, colind, val, opts, false);
    if (st != PSLR_OK) {
        fprintf(stderr, "pslr_setup: %s\n", c->err.c_str());
        pslr_destroy(c);
        return st;
    }
    *out = c;
    return PSLR_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- applies

// The per-CTA segment stream of one launch shape, built on first use: for
// CTA b and its subdomains b, b+grid, ..., the segments in exactly the order
// the kernel's consumers take them.  kind 0: apply (forward or transposed,
// with the low-rank term before the series when lr_before); kind 1: E_rr(m).
static pslr_status get_stream(pslr_ctx *c, OpSetHost &o, int kind, int m, bool lr_before,
                              const StreamDev **out) {
    char key[64];
    snprintf(key, sizeof(key), "%d/%d/%d", kind, m, (int)lr_before);
    auto it = o.streams.find(key);
    if (it != o.streams.end()) {
        *out = &it->second;
        return PSLR_OK;
    }
    const int s = c->s, G = o.grid;
    std::vector<StreamEnt> ent;
    std::vector<int64_t> off(G + 1, 0);
    auto add = [&](int i, std::initializer_list<int> cats) {
        for (int cat : cats) {
            int d = o.hsub[i];
            for (int k = 0; k < cat; ++k) d += o.hcnt[(size_t)kNCnt * i + k];
            for (int t = 0; t < o.hcnt[(size_t)kNCnt * i + cat]; ++t) {
                StreamEnt e;
                e.off = o.hdesc[d + t].off;
                e.bytes = o.hdesc[d + t].bytes;
                e.pad = 0;
                ent.push_back(e);
            }
        }
    };
    for (int b = 0; b < G; ++b) {
        off[b] = (int64_t)ent.size();
        if (kind == 0) {
            for (int i = b; i < s; i += G) {
                add(i, {kB1, kB2, kF});
                if (!lr_before) add(i, {kC1, kC2});
            }
            if (lr_before)
                for (int i = b; i < s; i += G) add(i, {kC1, kC2});
            for (int k = 1; k <= m; ++k)
                for (int i = b; i < s; i += G) add(i, {kE, kB1, kB2, kF, kCg, kC1, kC2});
            for (int i = b; i < s; i += G) add(i, {kE, kB1, kB2});
        } else {
            for (int rep = 0; rep <= m; ++rep) {
                for (int i = b; i < s; i += G) add(i, {kC1, kC2});
                for (int i = b; i < s; i += G) add(i, {kE, kB1, kB2, kF, kCg});
            }
        }
    }
    off[G] = (int64_t)ent.size();
    StreamDev sd;
    CK(upload(&sd.ent, ent));
    CK(upload(&sd.off, off));
    o.streams[key] = sd;
    *out = &o.streams[key];
    return PSLR_OK;
}

template <class T, class IO>
static void fill_params(pslr_ctx *c, ApplyParams<T, IO> &P, const OpSetHost &o, int dir, const StreamDev *sd) {
    P.segbase = o.seg;
    P.stream = sd->ent;
    P.stream_off = sd->off;
    P.cnt = o.cnt;
    P.ring = o.ring;
    P.slot_bytes = o.slot_bytes;
    P.pivot_post = dir;
    P.lowrank_after = dir;
    P.s = c->s;
    P.p = c->p;
    P.q = c->q;
    P.r = c->r;
    P.ldv = c->ldv;
    P.m = c->m;
    P.grid = o.grid;
    P.max_p = c->max_p;
    P.max_q = c->max_q;
    P.ioff = c->d_ioff;
    P.goff = c->d_goff;
    P.perm = c->d_perm;
    P.bpiv = c->d_bpiv;
    P.cpiv = c->d_cpiv;
    P.wbuf = reinterpret_cast<T *>(c->d_wbuf);
    P.acc = reinterpret_cast<T *>(c->d_acc);
    P.part = reinterpret_cast<T *>(c->d_part);
    P.bar = c->d_bar;
    P.err = c->d_err;
    P.skip = nullptr;
    P.wait_limit = c->wait_limit;
    P.rs = c->rs;
    P.omega = T(c->omega);
    P.dB = nullptr;
    P.dC = nullptr;
}

// Scratch of one apply launch: series iterates (2(q+1)), accumulator (q+1),
// per-subdomain partials (s*r), grid-barrier words (2) and the error word.
struct ApplyScratch {
    void *wbuf, *acc, *part;
    unsigned *bar;
    int *err;
};

static const StreamDev *find_stream(const OpSetHost &o, int kind, int m, bool lr_before) {
    char key[64];
    snprintf(key, sizeof(key), "%d/%d/%d", kind, m, (int)lr_before);
    auto it = o.streams.find(key);
    return it == o.streams.end() ? nullptr : &it->second;
}

// Precision forms of one apply launch: PSLR_FP64, PSLR_FP32, and (internal)
// kF32OnF64: FP32 arithmetic and BF16 V on FP64 input and output vectors, the
// FGMRES form with the FP32 preconditioner (no conversion kernels).
constexpr int kF32OnF64 = 2;

template <class T, class IO>
static void set_io(ApplyParams<T, IO> &P, const void *b, void *z, const int *skip, const ApplyScratch *scr) {
    P.b = static_cast<const IO *>(b);
    P.z = static_cast<IO *>(z);
    P.skip = skip;
    if (scr) {
        P.wbuf = static_cast<T *>(scr->wbuf);
        P.acc = static_cast<T *>(scr->acc);
        P.part = static_cast<T *>(scr->part);
        P.bar = scr->bar;
        P.err = scr->err;
    }
}

// The operator set an apply of this precision and direction runs on: the
// unit-diagonal set for forward FP64 applies where there is one.
static OpSetHost &apply_opset(pslr_ctx *c, int dir, int prec) {
    return dir == 0 && prec == 0 && c->has_unit ? c->ops_unit : c->ops[dir][prec];
}

static pslr_status apply_launch(pslr_ctx *c, const void *b, void *z, int form, int dir, const int *skip,
                                cudaStream_t st, const ApplyScratch *scr, bool may_allocate) {
    const int prec = form == PSLR_FP64 ? 0 : 1;  // operator set: FP64 or FP32 segments
    OpSetHost &o = apply_opset(c, dir, prec);
    const bool unit = &o == &c->ops_unit;
    const bool lr_before = c->r > 0 && dir == 0;
    const StreamDev *sd = find_stream(o, 0, c->m, lr_before);
    if (!sd) {
        if (!may_allocate)
            return fail(c, PSLR_ERR_STATE, "the segment stream of this launch shape is not built");
        pslr_status ss = get_stream(c, o, 0, c->m, lr_before, &sd);
        if (ss != PSLR_OK) return ss;
    }
    cudaError_t e;
    std::lock_guard<std::mutex> lock(g_launch_mutex);
    if (form == PSLR_FP64) {
        ApplyParams<double> P;
        fill_params(c, P, o, dir, sd);
        P.V = c->d_Vr;
        P.G = dir ? c->d_GT : c->d_G;
        set_io(P, b, z, skip, scr);
        if (unit) {
            P.dB = c->d_dB;
            P.dC = c->d_dC;
            e = launch_apply_fp64_unit(P, o.smem, o.dual, o.merged, st);
        } else {
            e = launch_apply_fp64(P, o.smem, o.dual, o.merged, st);
        }
    } else if (form == PSLR_FP32) {
        ApplyParams<float> P;
        fill_params(c, P, o, dir, sd);
        P.V = c->d_Vb;
        P.G = dir ? c->d_GTf : c->d_Gf;
        set_io(P, b, z, skip, scr);
        e = launch_apply_fp32(P, o.smem, o.dual, o.merged, st);
    } else {
        ApplyParams<float, double> P;
        fill_params(c, P, o, dir, sd);
        P.V = c->d_Vb;
        P.G = dir ? c->d_GTf : c->d_Gf;
        set_io(P, b, z, skip, scr);
        e = launch_apply_f32d(P, o.smem, o.dual, o.merged, st);
    }
    if (e != cudaSuccess) return fail(c, PSLR_ERR_CUDA, "apply launch: %s", cudaGetErrorString(e));
    return PSLR_OK;
}

static pslr_status apply_one(pslr_ctx *c, const void *b, void *z, int prec, int dir, const int *skip,
                             cudaStream_t st) {
    return apply_launch(c, b, z, prec, dir, skip, st, nullptr, true);
}

// Build the apply streams of the current (m, r) for both directions and
// precisions, so that no later apply has to allocate.
static pslr_status prebuild_streams(pslr_ctx *c) {
    for (int dir = 0; dir < 2; ++dir)
        for (int prec = 0; prec < 2; ++prec) {
            const StreamDev *sd = nullptr;
            pslr_status st = get_stream(c, apply_opset(c, dir, prec), 0, c->m, c->r > 0 && dir == 0, &sd);
            if (st != PSLR_OK) return st;
        }
    return PSLR_OK;
}

namespace pslr {
// Record an error on a context from another translation unit.
pslr_status report(pslr_ctx *c, pslr_status st, const char *msg) { return fail(c, st, "%s", msg); }

// Apply with caller-provided scratch and no allocation (used by the
// no-allocation entry point).  Returns PSLR_ERR_TOO_LARGE when the scratch
// does not hold this context's vectors.
pslr_status apply_with_scratch(pslr_ctx *c, const void *b, void *z, int prec, int dir, cudaStream_t st,
                               void *scratch, size_t scratch_bytes) {
    if (!c || !b || !z || !scratch || (prec != PSLR_FP64 && prec != PSLR_FP32))
        return fail(c, PSLR_ERR_ARG, "apply (no allocation): bad argument");
    const size_t head = 256;  // grid-barrier words
    const size_t need = head + sizeof(double) * ((size_t)3 * (c->q + 1) + (size_t)c->s * c->r);
    if (need > scratch_bytes)
        return fail(c, PSLR_ERR_TOO_LARGE,
                    "apply (no allocation): needs %zu bytes of scratch for q = %d, s = %d, r = %d; "
                    "the static scratch holds %zu",
                    need, c->q, c->s, c->r, scratch_bytes);
    char *p = static_cast<char *>(scratch);
    ApplyScratch scr;
    scr.bar = reinterpret_cast<unsigned *>(p);
    // the error word stays the context's own (allocated at set-up): pslr_sync
    // reads and clears it, and a latched error stops later applies of this
    // context, exactly as for pslr_apply
    scr.err = c->d_err;
    scr.wbuf = p + head;
    scr.acc = p + head + sizeof(double) * 2 * (c->q + 1);
    scr.part = p + head + sizeof(double) * 3 * (c->q + 1);
    // the shared array keeps the previous call's words (a call that gave up
    // leaves arrivals behind): the barrier starts at zero
    cudaError_t e = cudaMemsetAsync(p, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return fail(c, PSLR_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return apply_launch(c, b, z, prec, dir, nullptr, st, &scr, false);
}
}  // namespace pslr

static pslr_status apply_dir(pslr_ctx *c, const void *b, void *z, int32_t nrhs, pslr_prec prec, int dir,
                             void *stream) {
    if (!c || !b || !z || nrhs < 1 || (prec != PSLR_FP64 && prec != PSLR_FP32))
        return fail(c, PSLR_ERR_ARG, "apply: bad argument");
    const size_t es = prec == PSLR_FP64 ? 8 : 4;
    for (int j = 0; j < nrhs; ++j) {
        pslr_status st = apply_one(c, static_cast<const char *>(b) + j * es * c->n,
                                   static_cast<char *>(z) + j * es * c->n, prec, dir, nullptr,
                                   static_cast<cudaStream_t>(stream));
        if (st != PSLR_OK) return st;
    }
    return PSLR_OK;
}

// Algorithmic bytes of one forward apply (Algorithm 3) with this layout: each
// pass streams its segments once - m+2 B solves, m+1 C0 solves, m+1 passes of
// E and of F, m of C_g, 2 of V - plus the vectors each phase reads or writes
// (b gathered twice for f, once for g; z written once; per phase the
// interface iterate, accumulator and the C_g gathers).
static int64_t pslr_apply_bytes(const pslr_ctx *c, int prec) {
    const OpSetHost &o = c->ops[0][prec];
    const int64_t m = c->m, r = c->r, n = c->n, p = c->p, q = c->q;
    const int64_t vs = prec == 0 ? 8 : 4, vb = prec == 0 ? 8 : 2;
    int64_t b = (m + 2) * (o.cat_bytes[kB1] + o.cat_bytes[kB2]) +
                (m + 1) * (o.cat_bytes[kC1] + o.cat_bytes[kC2]) + (m + 1) * o.cat_bytes[kE] +
                (m + 1) * o.cat_bytes[kF] + m * o.cat_bytes[kCg];
    b += 2 * q * r * vb;
    int64_t vec = 2 * p + q + n;                // b reads, z write
    vec += (r > 0 ? 2 * q : 0) + 2 * q;         // t staging, w_0 and acc
    vec += m * (q + q + 2 * q);                 // per term: w_{k-1} read, w_k write, acc r/w
    b += vec * vs;
    return b;
}

extern "C" {

pslr_status pslr_apply(pslr_ctx *c, const void *b_dev, void *z_dev, int32_t nrhs, pslr_prec prec,
                       void *stream) {
    return apply_dir(c, b_dev, z_dev, nrhs, prec, 0, stream);
}

pslr_status pslr_apply_T(pslr_ctx *c, const void *b_dev, void *z_dev, int32_t nrhs, pslr_prec prec,
                         void *stream) {
    return apply_dir(c, b_dev, z_dev, nrhs, prec, 1, stream);
}

pslr_status pslr_sync(pslr_ctx *c, void *stream) {
    if (!c) return PSLR_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!c->h_err) CK(cudaMallocHost(&c->h_err, sizeof(int)));
    // the error word rides on the stream: one synchronisation, no blocking copy after it
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int e = *c->h_err;
    if (e != 0) {
        CK(cudaMemset(c->d_err, 0, sizeof(int)));
        CK(cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned)));
        return fail(c, static_cast<pslr_status>(e), "device reported: %s",
                    pslr_status_string(static_cast<pslr_status>(e)));
    }
    return PSLR_OK;
}

pslr_status pslr_apply_host(pslr_ctx *c, const void *b_host, void *z_host, int32_t nrhs, pslr_prec prec,
                            int32_t transpose, void *stream) {
    if (!c || !b_host || !z_host || nrhs < 1 || (prec != PSLR_FP64 && prec != PSLR_FP32))
        return fail(c, PSLR_ERR_ARG, "apply_host: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)(prec == PSLR_FP64 ? 8 : 4) * c->n * nrhs;
    if (bytes > c->io_bytes) {  // staging buffers owned by the context, grown on demand
        CK(cudaStreamSynchronize(st));
        cudaFree(c->d_io_b);
        cudaFree(c->d_io_z);
        c->d_io_b = c->d_io_z = nullptr;
        c->io_bytes = 0;
        CK(cudaMalloc(&c->d_io_b, bytes));
        CK(cudaMalloc(&c->d_io_z, bytes));
        c->io_bytes = bytes;
    }
    CK(cudaMemcpyAsync(c->d_io_b, b_host, bytes, cudaMemcpyHostToDevice, st));
    pslr_status s = apply_dir(c, c->d_io_b, c->d_io_z, nrhs, prec, transpose ? 1 : 0, stream);
    if (s == PSLR_OK) CK(cudaMemcpyAsync(z_host, c->d_io_z, bytes, cudaMemcpyDeviceToHost, st));
    pslr_status s2 = pslr_sync(c, stream);
    return s != PSLR_OK ? s : s2;
}

int64_t pslr_set_wait_limit(pslr_ctx *c, int64_t polls) {
    if (!c) return -1;
    int64_t old = c->wait_limit;
    if (polls != old) drop_graphs(c);
    c->wait_limit = polls;
    return old;
}

pslr_status pslr_get_maps(const pslr_ctx *c, int32_t *part, int32_t *is_interface, int32_t *perm) {
    if (!c) return PSLR_ERR_ARG;
    if (part) std::copy(c->part.begin(), c->part.end(), part);
    if (is_interface) std::copy(c->iface.begin(), c->iface.end(), is_interface);
    if (perm) std::copy(c->perm.begin(), c->perm.end(), perm);
    return PSLR_OK;
}

pslr_status pslr_get_info(const pslr_ctx *c, pslr_info *info) {
    if (!c || !info) return PSLR_ERR_ARG;
    pslr_info I;
    std::memset(&I, 0, sizeof(I));
    I.n = c->n;
    I.s = c->s;
    I.p = c->p;
    I.q = c->q;
    I.m = c->m;
    I.rank = c->r;
    I.nnz_A = c->nnz_A;
    I.nnz_ilu = c->nnz_ilu;
    I.nnz_lr = (int64_t)c->q * c->r + (int64_t)c->r * c->r;
    I.fill_ilu = (double)I.nnz_ilu / (double)I.nnz_A;
    I.fill_lr = (double)I.nnz_lr / (double)I.nnz_A;
    I.fill_total = I.fill_ilu + I.fill_lr;
    I.max_interior = c->max_p;
    I.max_interface = c->max_q;
    I.levels_B = c->levels_B;
    I.levels_C0 = c->levels_C;
    I.apply_bytes_fp64 = pslr_apply_bytes(c, 0);
    I.apply_bytes_fp32 = pslr_apply_bytes(c, 1);
    I.setup_threads = c->threads;
    I.layout_hash = c->layout_hash;
    I.layout_errors = c->layout_errors;
    I.omega = c->omega;
    I.nnz_fact_B = c->nnz_blk[0];
    I.nnz_fact_C0 = c->nnz_blk[1];
    I.nnz_E = c->nnz_blk[2];
    I.nnz_F = c->nnz_blk[3];
    I.nnz_Cg = c->nnz_blk[4];
    for (int prec = 0; prec < 2; ++prec) {
        I.grid[prec] = c->ops[0][prec].grid;
        I.ring[prec] = c->ops[0][prec].ring;
        I.ctas_per_sm[prec] = c->ops[0][prec].dual ? 2 : 1;
        I.merged[prec] = c->ops[0][prec].merged ? 1 : 0;
    }
    I.unit_sweeps = c->has_unit ? 1 : 0;
    I.device_factor = c->device_factor;
    I.factor_ms = c->factor_ms;
    *info = I;
    return PSLR_OK;
}

pslr_status pslr_plan(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
                      const pslr_opts *opts, int32_t m, int32_t rank, pslr_info *info, int32_t *part,
                      int32_t *is_interface, int32_t *perm) {
    TraceRange trace("pslr_plan");
    if (n <= 0 || !rowptr || !colind || !val || !opts || m < 0 || rank < 0) return PSLR_ERR_ARG;
    pslr_ctx *c = new pslr_ctx();
    pslr_status st = setup_impl(c, n, rowptr, colind, val, opts, true);
    if (st == PSLR_OK) {
        c->m = m;
        c->r = std::min(std::min<int>(rank, c->q), kMaxRank);
        if (info) pslr_get_info(c, info);
        pslr_get_maps(c, part, is_interface, perm);
    } else {
        fprintf(stderr, "pslr_plan: %s\n", c->err.c_str());
    }
    pslr_destroy(c);
    return st;
}

pslr_status pslr_grad_values(pslr_ctx *c, const double *lambda_dev, const double *u_dev, double *grad_dev,
                             void *stream) {
    if (!c || !lambda_dev || !u_dev || !grad_dev) return fail(c, PSLR_ERR_ARG, "grad_values: bad argument");
    launch_grad_values(c->n, c->d_rp, c->d_ci, lambda_dev, u_dev, grad_dev, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return PSLR_OK;
}

pslr_status pslr_matvec(pslr_ctx *c, const double *x_dev, double *y_dev, int32_t transpose, void *stream) {
    if (!c || !x_dev || !y_dev) return fail(c, PSLR_ERR_ARG, "matvec: bad argument");
    launch_residual(c->n, transpose ? c->d_rpT : c->d_rp, transpose ? c->d_ciT : c->d_ci,
                    transpose ? c->d_avT : c->d_av, x_dev, nullptr, y_dev, static_cast<cudaStream_t>(stream));
    CK(cudaGetLastError());
    return PSLR_OK;
}

}  // extern "C"

// ------------------------------------------------------------ low-rank term

// G = (I - H)^{-1} - I by LU with partial pivoting of I - H (Eq. 3.17).
// H and G are r x r column-major.  Returns false if I - H is singular.
static bool compute_G(int r, const std::vector<double> &H, std::vector<double> &G) {
    std::vector<double> a((size_t)r * r);
    double amax = 0.0;
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            a[(size_t)i * r + j] = (i == j ? 1.0 : 0.0) - H[(size_t)j * r + i];
            amax = std::max(amax, std::fabs(a[(size_t)i * r + j]));
        }
    std::vector<int> perm(r);
    for (int i = 0; i < r; ++i) perm[i] = i;
    for (int k = 0; k < r; ++k) {
        int pr = k;
        double best = std::fabs(a[(size_t)k * r + k]);
        for (int i = k + 1; i < r; ++i)
            if (std::fabs(a[(size_t)i * r + k]) > best) {
                best = std::fabs(a[(size_t)i * r + k]);
                pr = i;
            }
        if (!(best > 1e-14 * amax)) return false;
        if (pr != k) {
            for (int j = 0; j < r; ++j) std::swap(a[(size_t)k * r + j], a[(size_t)pr * r + j]);
            std::swap(perm[k], perm[pr]);
        }
        for (int i = k + 1; i < r; ++i) {
            double l = a[(size_t)i * r + k] / a[(size_t)k * r + k];
            a[(size_t)i * r + k] = l;
            for (int j = k + 1; j < r; ++j) a[(size_t)i * r + j] -= l * a[(size_t)k * r + j];
        }
    }
    G.assign((size_t)r * r, 0.0);
    std::vector<double> x(r);
    for (int j = 0; j < r; ++j) {
        for (int i = 0; i < r; ++i) x[i] = (perm[i] == j) ? 1.0 : 0.0;
        for (int i = 0; i < r; ++i)
            for (int l = 0; l < i; ++l) x[i] -= a[(size_t)i * r + l] * x[l];
        for (int i = r - 1; i >= 0; --i) {
            for (int l = i + 1; l < r; ++l) x[i] -= a[(size_t)i * r + l] * x[l];
            x[i] /= a[(size_t)i * r + i];
        }
        for (int i = 0; i < r; ++i) G[(size_t)j * r + i] = x[i] - (i == j ? 1.0 : 0.0);
    }
    return true;
}

// Install V (device FP64 q x r, already in c->d_V) plus host G: derived copies
// (row-major FP64 and BF16 V for the apply, G^T, FP32 G and G^T).
static pslr_status install_lowrank(pslr_ctx *c, int m, int r, const std::vector<double> &G) {
    const int q = c->q;
    ++c->lr_gen;
    drop_graphs(c);
    c->m = m;
    c->r = r;
    c->G = G;
    c->omega = 1.0;
    cudaFree(c->d_Vr); cudaFree(c->d_Vb); cudaFree(c->d_G); cudaFree(c->d_GT); cudaFree(c->d_Gf); cudaFree(c->d_GTf);
    cudaFree(c->d_part);
    c->d_Vr = nullptr; c->d_Vb = nullptr; c->d_G = c->d_GT = nullptr; c->d_Gf = c->d_GTf = nullptr; c->d_part = nullptr;
    c->ldv = 0;
    {
        pslr_status ps = plan_launch(c);
        if (ps != PSLR_OK) return ps;
    }
    if (r == 0) return prebuild_streams(c);
    c->V.resize((size_t)q * r);
    CK(cudaMemcpy(c->V.data(), c->d_V, sizeof(double) * (size_t)q * r, cudaMemcpyDeviceToHost));
    c->ldv = (r + 7) & ~7;
    std::vector<double> vr((size_t)q * c->ldv, 0.0);
    std::vector<uint16_t> vb((size_t)q * c->ldv, 0);
    for (int col = 0; col < r; ++col)
        for (int i = 0; i < q; ++i) {
            const double v = c->V[(size_t)col * q + i];
            vr[(size_t)i * c->ldv + col] = v;
            vb[(size_t)i * c->ldv + col] = f32_to_bf16((float)v);
        }
    std::vector<double> GT((size_t)r * r);
    std::vector<float> Gf((size_t)r * r), GTf((size_t)r * r);
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            GT[(size_t)j * r + i] = G[(size_t)i * r + j];
            Gf[(size_t)j * r + i] = (float)G[(size_t)j * r + i];
            GTf[(size_t)j * r + i] = (float)G[(size_t)i * r + j];
        }
    CK(upload(&c->d_Vr, vr));
    CK(upload(&c->d_Vb, vb));
    CK(upload(&c->d_G, G));
    CK(upload(&c->d_GT, GT));
    CK(upload(&c->d_Gf, Gf));
    CK(upload(&c->d_GTf, GTf));
    CK(cudaMalloc(&c->d_part, sizeof(double) * (size_t)c->s * r + 16));
    return prebuild_streams(c);
}

extern "C" {

pslr_status pslr_set_neumann(pslr_ctx *c, int32_t m, double omega, void *stream) {
    if (!c || m < 0 || !(omega > 0.0) || !std::isfinite(omega))
        return fail(c, PSLR_ERR_ARG, "set_neumann: bad argument (m >= 0, omega > 0)");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    free_lowrank(c);
    pslr_status st = install_lowrank(c, m, 0, {});
    if (st != PSLR_OK) return st;
    c->omega = omega;  // install_lowrank dropped the captured cycles
    return PSLR_OK;
}

pslr_status pslr_set_lowrank(pslr_ctx *c, int32_t m, int32_t rank, const double *V, const double *G,
                             void *stream) {
    if (!c || m < 0 || rank < 0 || rank > kMaxRank || rank > c->q || (rank > 0 && (!V || !G)))
        return fail(c, PSLR_ERR_ARG, "set_lowrank: bad argument (rank must be <= %d and <= q)", kMaxRank);
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    free_lowrank(c);
    if (rank > 0) {
        CK(cudaMalloc(&c->d_V, sizeof(double) * (size_t)c->q * rank));
        CK(cudaMemcpy(c->d_V, V, sizeof(double) * (size_t)c->q * rank, cudaMemcpyHostToDevice));
    }
    std::vector<double> g(G, G + (size_t)rank * rank);
    pslr_status st = install_lowrank(c, m, rank, g);
    if (st == PSLR_OK) c->H.clear();
    return st;
}

pslr_status pslr_get_lowrank(const pslr_ctx *c, double *V, double *H, double *G) {
    if (!c) return PSLR_ERR_ARG;
    if (V && c->r) std::copy(c->V.begin(), c->V.end(), V);
    if (H && c->r && !c->H.empty()) std::copy(c->H.begin(), c->H.end(), H);
    if (G && c->r) std::copy(c->G.begin(), c->G.end(), G);
    return PSLR_OK;
}

}  // extern "C"

static pslr_status kwork_alloc(pslr_ctx *c, KWork &W, int len, int kcols) {
    W.nblk = krylov_blocks(len);
    CK(cudaMalloc(&W.part, sizeof(double) * krylov_part_doubles(W.nblk, kcols + 1)));
    CK(cudaMalloc(&W.h1, sizeof(double) * (kcols + 1)));
    CK(cudaMalloc(&W.h2, sizeof(double) * (kcols + 1)));
    CK(cudaMalloc(&W.wn2, sizeof(double) * 2));
    CK(cudaMalloc(&W.hn, sizeof(double) * 2));
    CK(cudaMalloc(&W.ticket, sizeof(unsigned) * krylov_tickets()));
    CK(cudaMemset(W.ticket, 0, sizeof(unsigned) * krylov_tickets()));
    return PSLR_OK;
}

static void kwork_free(KWork &W) {
    cudaFree(W.part); cudaFree(W.h1); cudaFree(W.h2); cudaFree(W.wn2); cudaFree(W.hn); cudaFree(W.ticket);
    W = KWork();
}

// w <- w - V(:,0:k)(V^T w) twice (CGS2); h (device) = summed coefficients,
// wn2 = ||w||^2.  With k == 0 only the norm is taken.
static void cgs2(KWork &W, int len, int k, const double *V, int64_t ld, double *w, const int32_t *rp,
                 const int32_t *ci, const double *av, const double *z, const int *skip, cudaStream_t st) {
    if (k > 0) {
        launch_cgs_pass(len, k, V, ld, w, nullptr, 0, W.part, W.h1, W.ticket, rp, ci, av, z, skip, st);
        launch_cgs_pass(len, k, V, ld, w, W.h1, 0, W.part, W.h2, W.ticket, nullptr, nullptr, nullptr,
                        nullptr, skip, st);
        launch_cgs_pass(len, k, V, ld, w, W.h2, 1, W.part, W.wn2, W.ticket, nullptr, nullptr, nullptr,
                        nullptr, skip, st);
    } else {
        launch_cgs_pass(len, 0, V, ld, w, nullptr, 1, W.part, W.wn2, W.ticket, rp, ci, av, z, skip, st);
    }
}

static pslr_status launch_err(pslr_ctx *c, const double *vin, double *vout, int m, cudaStream_t st) {
    OpSetHost &o = c->ops[0][0];
    const StreamDev *sd = nullptr;
    pslr_status ss = get_stream(c, o, 1, m, false, &sd);
    if (ss != PSLR_OK) return ss;
    ErrParams<double> P;
    P.segbase = o.seg;
    P.stream = sd->ent;
    P.stream_off = sd->off;
    P.cnt = o.cnt;
    P.ring = o.ring;
    P.slot_bytes = o.slot_bytes;
    P.s = c->s;
    P.p = c->p;
    P.q = c->q;
    P.m = m;
    P.grid = o.grid;
    P.max_p = c->max_p;
    P.max_q = c->max_q;
    P.ioff = c->d_ioff;
    P.goff = c->d_goff;
    P.bpiv = c->d_bpiv;
    P.cpiv = c->d_cpiv;
    P.vin = vin;
    P.vout = vout;
    P.abuf = c->d_eab;
    P.bar = c->d_bar;
    P.err = c->d_err;
    P.wait_limit = c->wait_limit;
    P.rs = c->rs;
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lock(g_launch_mutex);
        e = launch_err_fp64(P, o.smem, o.dual, o.merged, st);
    }
    if (e != cudaSuccess) return fail(c, PSLR_ERR_CUDA, "E_rr launch: %s", cudaGetErrorString(e));
    return PSLR_OK;
}

extern "C" {

pslr_status pslr_build_lowrank(pslr_ctx *c, int32_t m, int32_t rank, int32_t full_rank, void *stream) {
    TraceRange trace("pslr_build_lowrank");
    if (!c || m < 0 || rank < 0) return fail(c, PSLR_ERR_ARG, "build_lowrank: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(st));
    free_lowrank(c);
    const int q = c->q;
    if (rank > q) rank = q;
    if (rank > kMaxRank) return fail(c, PSLR_ERR_ARG, "rank must be <= %d", kMaxRank);
    c->m = m;
    if (rank == 0) return install_lowrank(c, m, 0, {});
    const int r = rank;
    double *Vq = nullptr, *w = nullptr;
    CK(cudaMalloc(&Vq, sizeof(double) * (size_t)q * (r + 1)));
    CK(cudaMalloc(&w, sizeof(double) * (size_t)q));
    KWork W;
    pslr_status ks = kwork_alloc(c, W, q, r + 1);
    auto cleanup = [&]() {
        cudaFree(w);
        kwork_free(W);
    };
    if (ks != PSLR_OK) {
        cudaFree(Vq);
        cleanup();
        return ks;
    }
    std::vector<double> Hb((size_t)(r + 1) * r, 0.0);  // (r+1) x r column-major
    double hn = 0.0, hf2 = 0.0;
    int kept = r, tvec = 0;
    pslr_status status = PSLR_OK;
    // v_1 = u / ||u||, u = SplitMix64 draws
    launch_splitmix(q, c->seed, 0, Vq, st);
    cgs2(W, q, 0, Vq, q, Vq, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    {
        double u2 = 0.0;
        CK(cudaMemcpyAsync(&u2, W.wn2, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double un = std::sqrt(u2);
        CK(cudaMemcpyAsync(W.hn, &un, sizeof(double), cudaMemcpyHostToDevice, st));
        launch_normalize(q, Vq, Vq, W.hn, nullptr, st);
    }
    std::vector<double> hcol(r + 2);
    for (int j = 0; j < r; ++j) {
        pslr_status es = launch_err(c, Vq + (size_t)j * q, w, m, st);
        if (es != PSLR_OK) { status = es; break; }
        cgs2(W, q, j + 1, Vq, q, w, nullptr, nullptr, nullptr, nullptr, nullptr, st);
        CK(cudaMemcpyAsync(hcol.data(), W.h1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
        std::vector<double> h2(j + 1);
        CK(cudaMemcpyAsync(h2.data(), W.h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
        double wn2 = 0.0;
        CK(cudaMemcpyAsync(&wn2, W.wn2, sizeof(double), cudaMemcpyDeviceToHost, st));
        pslr_status ss = pslr_sync(c, stream);
        if (ss != PSLR_OK) { status = ss; break; }
        hn = std::sqrt(wn2);
        for (int i = 0; i <= j; ++i) {
            double h = hcol[i] + h2[i];
            Hb[(size_t)j * (r + 1) + i] = h;
            hf2 += h * h;
        }
        hf2 += wn2;
        if (!std::isfinite(hn) || !std::isfinite(hf2)) { status = fail(c, PSLR_ERR_NAN, "NaN in Arnoldi"); break; }
        if (j == r - 1) break;
        if (hn <= 1e-12 * std::sqrt(hf2)) {
            if (!full_rank) {
                kept = j + 1;
                status = PSLR_ERR_BREAKDOWN;
                break;
            }
            ++tvec;
            double *vn = Vq + (size_t)(j + 1) * q;
            launch_splitmix(q, c->seed, (uint64_t)tvec * q, vn, st);
            cgs2(W, q, j + 1, Vq, q, vn, nullptr, nullptr, nullptr, nullptr, nullptr, st);
            double nn2 = 0.0;
            CK(cudaMemcpyAsync(&nn2, W.wn2, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double nn = std::sqrt(nn2);
            CK(cudaMemcpyAsync(W.hn, &nn, sizeof(double), cudaMemcpyHostToDevice, st));
            launch_normalize(q, vn, vn, W.hn, nullptr, st);
            Hb[(size_t)j * (r + 1) + j + 1] = 0.0;
        } else {
            Hb[(size_t)j * (r + 1) + j + 1] = hn;
            CK(cudaMemcpyAsync(W.hn, &hn, sizeof(double), cudaMemcpyHostToDevice, st));
            launch_normalize(q, w, Vq + (size_t)(j + 1) * q, W.hn, nullptr, st);
        }
    }
    CK(cudaStreamSynchronize(st));
    cleanup();
    if (status != PSLR_OK && status != PSLR_ERR_BREAKDOWN) {
        cudaFree(Vq);
        return status;
    }
    std::vector<double> H((size_t)kept * kept), G;
    for (int j = 0; j < kept; ++j)
        for (int i = 0; i < kept; ++i) H[(size_t)j * kept + i] = Hb[(size_t)j * (r + 1) + i];
    if (!compute_G(kept, H, G)) {
        cudaFree(Vq);
        return fail(c, PSLR_ERR_SINGULAR_IMH, "I - H is singular");
    }
    c->d_V = Vq;  // first `kept` columns (leading dimension q)
    pslr_status st2 = install_lowrank(c, m, kept, G);
    if (st2 != PSLR_OK) return st2;
    c->H = H;
    if (status == PSLR_ERR_BREAKDOWN)
        return fail(c, PSLR_ERR_BREAKDOWN, "Arnoldi breakdown: rank truncated to %d", kept);
    return PSLR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------- FGMRES

static pslr_status krylov_alloc(pslr_ctx *c, int restart) {
    if (c->kr_restart == restart) return PSLR_OK;
    free_krylov(c);
    const size_t n = c->n;
    CK(cudaMalloc(&c->d_kV, sizeof(double) * n * (restart + 1)));
    CK(cudaMalloc(&c->d_kZ, sizeof(double) * n * restart));
    CK(cudaMalloc(&c->d_kw, sizeof(double) * n));
    CK(cudaMalloc(&c->d_kr, sizeof(double) * n));
    CK(cudaMalloc(&c->d_kH, sizeof(double) * (restart + 1) * restart));
    CK(cudaMalloc(&c->d_krot, sizeof(double) * 2 * (restart + 1)));
    CK(cudaMalloc(&c->d_kgam, sizeof(double) * (restart + 1)));
    CK(cudaMalloc(&c->d_kstate, sizeof(int) * 2));
    CK(cudaMalloc(&c->d_kskip, sizeof(int)));
    CK(cudaMalloc(&c->d_ktol, sizeof(double)));
    pslr_status ks = kwork_alloc(c, c->kw, (int)n, restart + 1);
    if (ks != PSLR_OK) return ks;
    if (!c->kcap) CK(cudaStreamCreateWithFlags(&c->kcap, cudaStreamNonBlocking));
    c->kr_restart = restart;
    return PSLR_OK;
}

// The Arnoldi steps j = 0 .. k-1 of one restart cycle (Section 4): apply the
// preconditioner to v_j (the FP32 form reads and writes the FP64 vectors),
// orthogonalise A z_j against V by CGS2, update H, the Givens rotations and
// gamma, and normalise v_{j+1}.  Once the Hessenberg kernel meets the
// tolerance it raises the skip flag and every later kernel of the cycle
// returns at once, so a full cycle can be enqueued (or replayed) blind.
static pslr_status enqueue_arnoldi(pslr_ctx *c, int j0, int j1, int prec, int dir, cudaStream_t st) {
    const int n = c->n, k = c->kr_restart;
    const int32_t *rp = dir ? c->d_rpT : c->d_rp, *ci = dir ? c->d_ciT : c->d_ci;
    const double *av = dir ? c->d_avT : c->d_av;
    KWork &W = c->kw;
    for (int j = j0; j < j1; ++j) {
        double *vj = c->d_kV + (size_t)j * n, *zj = c->d_kZ + (size_t)j * n;
        pslr_status a;
        a = apply_one(c, vj, zj, prec == PSLR_FP64 ? (int)PSLR_FP64 : kF32OnF64, dir, c->d_kskip, st);
        if (a != PSLR_OK) return a;
        cgs2(W, n, j + 1, c->d_kV, n, c->d_kw, rp, ci, av, zj, c->d_kskip, st);
        launch_hess_normalize(j, W.h1, W.h2, W.wn2, c->d_kH, k + 1, c->d_krot, c->d_kgam, c->d_ktol, c->d_kstate,
                              c->d_kskip, n, c->d_kw, c->d_kV + (size_t)(j + 1) * n, st);
    }
    return PSLR_OK;
}

// A full restart cycle as a CUDA graph, captured once per (precision,
// direction) on the context's private stream; nullptr when capture fails
// (the caller then launches the cycle directly).
static cudaGraphExec_t arnoldi_graph(pslr_ctx *c, int prec, int dir) {
    const auto key = std::make_pair(prec, dir);
    auto it = c->kgraphs.find(key);
    if (it != c->kgraphs.end()) return it->second;
    // the apply's segment stream must exist before capture: building it allocates
    const StreamDev *sd = nullptr;
    if (get_stream(c, apply_opset(c, dir, prec == PSLR_FP64 ? 0 : 1), 0, c->m, c->r > 0 && dir == 0, &sd) !=
        PSLR_OK)
        return nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    if (cudaStreamBeginCapture(c->kcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const pslr_status st = enqueue_arnoldi(c, 0, c->kr_restart, prec, dir, c->kcap);
    const cudaError_t e = cudaStreamEndCapture(c->kcap, &g);
    if (st != PSLR_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) x = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (x) c->kgraphs[key] = x;
    return x;
}

extern "C" {

pslr_status pslr_solve(pslr_ctx *c, const double *b_dev, double *x_dev, double rtol, int32_t restart,
                       int32_t maxit, pslr_prec prec, int32_t transpose, int32_t *iters, double *relres,
                       void *stream) {
    TraceRange trace("pslr_solve");
    if (!c || !b_dev || !x_dev || restart < 1 || restart > 127 || maxit < 0 || !(rtol > 0.0) ||
        (prec != PSLR_FP64 && prec != PSLR_FP32))
        return fail(c, PSLR_ERR_ARG, "solve: bad argument (restart must be 1..127)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pslr_status as = krylov_alloc(c, restart);
    if (as != PSLR_OK) return as;
    const int n = c->n, k = restart;
    const int dir = transpose ? 1 : 0;
    const int32_t *rp = dir ? c->d_rpT : c->d_rp, *ci = dir ? c->d_ciT : c->d_ci;
    const double *av = dir ? c->d_avT : c->d_av;
    KWork &W = c->kw;
    int its = 0;
    double bn2 = 0.0;
    cgs2(W, n, 0, nullptr, n, const_cast<double *>(b_dev), nullptr, nullptr, nullptr, nullptr, nullptr, st);
    CK(cudaMemcpyAsync(&bn2, W.wn2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, st));
    pslr_status ss = pslr_sync(c, stream);
    if (ss != PSLR_OK) return ss;
    const double bn = std::sqrt(bn2);
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    if (bn == 0.0) return PSLR_OK;
    if (!std::isfinite(bn)) return fail(c, PSLR_ERR_NAN, "right-hand side is not finite");
    const double tol_abs = rtol * bn;
    CK(cudaMemcpyAsync(c->d_ktol, &tol_abs, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_kr, b_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rn = bn;
    std::vector<double> H((size_t)(k + 1) * k), gam(k + 1), y(k);
    pslr_status result = PSLR_ERR_NOT_CONVERGED;
    while (its < maxit) {
        // v_1 = r / ||r||, gamma = ||r|| e_1
        std::vector<double> g0(k + 1, 0.0);
        g0[0] = rn;
        CK(cudaMemcpyAsync(c->d_kgam, g0.data(), sizeof(double) * (k + 1), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(W.hn, &rn, sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(c->d_kstate, 0, sizeof(int) * 2, st));
        CK(cudaMemsetAsync(c->d_kskip, 0, sizeof(int), st));
        launch_normalize(n, c->d_kr, c->d_kV, W.hn, nullptr, st);
        CK(cudaStreamSynchronize(st));
        const int jmax = std::min(k, maxit - its);
        cudaGraphExec_t g = jmax == k ? arnoldi_graph(c, prec, dir) : nullptr;
        if (g) {
            CK(cudaGraphLaunch(g, st));
        } else {
            pslr_status a = enqueue_arnoldi(c, 0, jmax, prec, dir, st);
            if (a != PSLR_OK) return a;
        }
        int state[2] = {0, 0};
        CK(cudaMemcpyAsync(state, c->d_kstate, sizeof(state), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(H.data(), c->d_kH, sizeof(double) * (k + 1) * k, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(gam.data(), c->d_kgam, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
        ss = pslr_sync(c, stream);
        if (ss != PSLR_OK) return ss;
        const int jd = state[0];
        its += jd;
        // H(0:jd, 0:jd) y = gamma(0:jd): upper triangular after the rotations
        for (int i = jd - 1; i >= 0; --i) {
            double a = gam[i];
            for (int l = i + 1; l < jd; ++l) a -= H[(size_t)l * (k + 1) + i] * y[l];
            y[i] = a / H[(size_t)i * (k + 1) + i];
        }
        bool finite = true;
        for (int i = 0; i < jd; ++i) finite &= std::isfinite(y[i]);
        if (!finite) return fail(c, PSLR_ERR_NAN, "NaN in the FGMRES least-squares solution");
        CK(cudaMemcpyAsync(W.h1, y.data(), sizeof(double) * std::max(jd, 1), cudaMemcpyHostToDevice, st));
        launch_gemv_add(n, jd, c->d_kZ, n, W.h1, x_dev, st);
        launch_residual(n, rp, ci, av, x_dev, b_dev, c->d_kr, st);
        cgs2(W, n, 0, nullptr, n, c->d_kr, nullptr, nullptr, nullptr, nullptr, nullptr, st);
        double rn2 = 0.0;
        CK(cudaMemcpyAsync(&rn2, W.wn2, sizeof(double), cudaMemcpyDeviceToHost, st));
        ss = pslr_sync(c, stream);
        if (ss != PSLR_OK) return ss;
        rn = std::sqrt(rn2);
        if (!std::isfinite(rn)) return fail(c, PSLR_ERR_NAN, "residual is not finite");
        if (rn <= rtol * bn) {
            result = PSLR_OK;
            break;
        }
        if (jd == 0) break;
    }
    if (iters) *iters = its;
    if (relres) *relres = rn / bn;
    if (result != PSLR_OK) return fail(c, PSLR_ERR_NOT_CONVERGED, "FGMRES reached maxit = %d", maxit);
    return PSLR_OK;
}

}  // extern "C"

// ------------------------------------------------------ view for the batch

namespace pslr {

bool sys_export(const pslr_ctx *c, SysExport *e) {
    if (!c || !c->ops[0][0].seg || !c->ops[0][1].seg) return false;
    e->n = c->n;
    e->s = c->s;
    e->p = c->p;
    e->q = c->q;
    e->m = c->m;
    e->r = c->r;
    e->factor = c->factor;
    e->max_p = c->max_p;
    e->max_q = c->max_q;
    e->ioff = c->d_ioff;
    e->goff = c->d_goff;
    e->perm = c->d_perm;
    e->rp = c->d_rp;
    e->ci = c->d_ci;
    e->av = c->d_av;
    e->V = c->d_Vr;
    e->Vb = c->d_Vb;
    e->ldv = c->ldv;
    e->G = c->d_G;
    e->Gf = c->d_Gf;
    for (int prec = 0; prec < 2; ++prec) {
        e->seg[prec] = c->ops[0][prec].seg;
        e->cnt[prec] = c->ops[0][prec].cnt;
        e->slot_bytes[prec] = c->ops[0][prec].slot_bytes;
        e->seg_bytes[prec] = c->ops[0][prec].seg_total;
    }
    e->lr_gen = c->lr_gen;
    e->omega = c->omega;
    e->ioff_h = c->ioff;
    e->goff_h = c->goff;
    return true;
}

void sys_segments(const pslr_ctx *c, int prec, int i, int cat, int64_t shift, std::vector<StreamEnt> &out) {
    const OpSetHost &o = c->ops[0][prec];
    int d = o.hsub[i];
    for (int k = 0; k < cat; ++k) d += o.hcnt[(size_t)kNCnt * i + k];
    for (int t = 0; t < o.hcnt[(size_t)kNCnt * i + cat]; ++t) {
        StreamEnt e;
        e.off = o.hdesc[d + t].off + shift;
        e.bytes = o.hdesc[d + t].bytes;
        e.pad = 0;
        out.push_back(e);
    }
}

uint64_t sys_lr_gen(const pslr_ctx *c) { return c ? c->lr_gen : 0; }

}  // namespace pslr
