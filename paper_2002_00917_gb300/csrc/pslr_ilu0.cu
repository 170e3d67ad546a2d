// ILU(0) local factors on the device (Algorithm 1, steps 3-4, with ILU(0) as
// the local factorization), for the set-up (pslr_opts.device_factor) and as
// the C entry point pslr_ilu0_device.
//
// The matrix is block diagonal, as B = blockdiag(B_i) and C0 = blockdiag(C_i)
// are (Eq. 2.1, Eq. 3.1), and ILU(0) runs in the IKJ order (Saad, Iterative
// Methods, Sec. 10.3.2): for row i and every stored column k < i, in
// ascending order, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for every j > k
// stored in row i and in row k.  Row i reads only the rows k < i it stores,
// so the rows of one level of that dependency graph - the level sets of the
// L sweep - are independent.  One CTA per diagonal block walks the block's
// levels with a CTA barrier between them, one thread per row; a thread
// writes only its own row, and the rows it reads were finished at earlier
// levels.  Matching j in rows i and k is a merge of two ascending column
// lists, so no thread needs a dense scatter array.
//
// No waits: every loop is bounded by the pattern, which the host checks
// before anything is copied to the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <string>
#include <vector>

#include "pslr.h"

namespace pslr {

namespace {

constexpr int kIluThreads = 256;

struct Ilu0Params {
    const int32_t *rp, *ci;  // CSR pattern, global row and column numbers
    const int32_t *dg;       // position of each row's diagonal entry
    double *v;               // values, factored in place
    const int32_t *rows;     // the rows of every block, level by level
    const int32_t *lptr;     // level l holds rows[lptr[l] .. lptr[l+1])
    const int32_t *blev;     // block b holds levels blev[b] .. blev[b+1]
    int nb;
    int *bad;                // smallest row that met a zero pivot, INT_MAX if none
};

// Row i of the IKJ elimination; every row k it reads is final.
__device__ void ilu0_row(const Ilu0Params &P, int i) {
    const int a1 = P.rp[i + 1], di = P.dg[i];
    for (int k = P.rp[i]; k < di; ++k) {
        const int kk = P.ci[k];
        const int dk = P.dg[kk];
        const double piv = P.v[dk];
        if (piv == 0.0) {  // row kk has reported itself; nothing to divide by
            atomicMin(P.bad, i);
            return;
        }
        const double l = P.v[k] / piv;
        P.v[k] = l;
        // j > kk: row kk's U entries after its diagonal against row i's
        // entries after column kk, both ascending
        int t = dk + 1, u = k + 1;
        const int t1 = P.rp[kk + 1];
        while (t < t1 && u < a1) {
            const int cj = P.ci[t], cu = P.ci[u];
            if (cj == cu) {
                P.v[u] = fma(-l, P.v[t], P.v[u]);
                ++t;
                ++u;
            } else if (cj < cu) {
                ++t;
            } else {
                ++u;
            }
        }
    }
    if (P.v[di] == 0.0) atomicMin(P.bad, i);
}

__global__ void __launch_bounds__(kIluThreads) k_ilu0_levels(const Ilu0Params P) {
    for (int b = blockIdx.x; b < P.nb; b += gridDim.x) {
        for (int l = P.blev[b]; l < P.blev[b + 1]; ++l) {
            for (int t = P.lptr[l] + (int)threadIdx.x; t < P.lptr[l + 1]; t += kIluThreads) ilu0_row(P, P.rows[t]);
            __syncthreads();  // level l complete (and visible) before level l + 1 reads it
        }
    }
}

// Host check of the pattern and the level sets: returns an empty string when
// the pattern is valid, else the reason.
std::string ilu0_levels(int n, int nb, const int32_t *bptr, const int32_t *rp, const int32_t *ci,
                        std::vector<int32_t> &dg, std::vector<int32_t> &rows, std::vector<int32_t> &lptr,
                        std::vector<int32_t> &blev) {
    char msg[160];
    if (bptr[0] != 0 || bptr[nb] != n) return "block_ptr must start at 0 and end at n";
    for (int b = 0; b < nb; ++b)
        if (bptr[b + 1] < bptr[b]) return "block_ptr not monotone";
    if (rp[0] != 0) return "rowptr[0] != 0";
    dg.assign(n, -1);
    std::vector<int32_t> lev(n, 0);
    rows.resize(n);
    lptr.assign(1, 0);
    blev.assign(1, 0);
    std::vector<int32_t> cnt;
    for (int b = 0; b < nb; ++b) {
        const int r0 = bptr[b], r1 = bptr[b + 1];
        int depth = 0;
        for (int i = r0; i < r1; ++i) {
            if (rp[i + 1] < rp[i]) {
                snprintf(msg, sizeof msg, "rowptr not monotone at row %d", i);
                return msg;
            }
            int lv = 0;
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int j = ci[k];
                if (j < r0 || j >= r1) {
                    snprintf(msg, sizeof msg, "row %d: column %d outside its diagonal block [%d, %d)", i, j, r0, r1);
                    return msg;
                }
                if (k > rp[i] && ci[k - 1] >= j) {
                    snprintf(msg, sizeof msg, "row %d: columns not strictly ascending", i);
                    return msg;
                }
                if (j == i) dg[i] = k;
                if (j < i) lv = std::max(lv, lev[j] + 1);
            }
            if (dg[i] < 0) {
                snprintf(msg, sizeof msg, "row %d holds no diagonal entry", i);
                return msg;
            }
            lev[i] = lv;
            depth = std::max(depth, lv + 1);
        }
        // rows of the block by level, ascending row number within a level
        cnt.assign(depth + 1, 0);
        for (int i = r0; i < r1; ++i) ++cnt[lev[i] + 1];
        for (int l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
        for (int l = 1; l <= depth; ++l) lptr.push_back(r0 + cnt[l]);
        for (int i = r0; i < r1; ++i) rows[r0 + cnt[lev[i]]++] = i;
        blev.push_back((int32_t)lptr.size() - 1);
    }
    return std::string();
}

template <class T>
cudaError_t upload(T *&d, const T *h, size_t count, cudaStream_t st) {
    cudaError_t e = cudaMalloc(&d, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) return e;
    return count == 0 ? cudaSuccess : cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, st);
}
template <class T>
cudaError_t upload(T *&d, const std::vector<T> &h, cudaStream_t st) {
    return upload(d, h.data(), h.size(), st);
}

}  // namespace

// ILU(0) of blockdiag(M_0 .. M_{nb-1}) (rows bptr[b] .. bptr[b+1] form block
// b) on the device: the host pattern rp / ci is checked (columns ascending,
// inside the row's block, diagonal present), its level sets computed, and
// val_dev factored in place on stream st.  On PSLR_ERR_ZERO_PIVOT *bad_row is
// the first row (in row order) whose pivot is zero.  *kernel_ms (if not null)
// receives the factorization kernel's time.  why explains a failure.
pslr_status ilu0_device_blocks(int n, int nb, const int32_t *bptr, const int32_t *rp, const int32_t *ci,
                               double *val_dev, cudaStream_t st, float *kernel_ms, int *bad_row,
                               std::string &why) {
    if (bad_row) *bad_row = -1;
    if (kernel_ms) *kernel_ms = 0.f;
    std::vector<int32_t> dg, rows, lptr, blev;
    why = ilu0_levels(n, nb, bptr, rp, ci, dg, rows, lptr, blev);
    if (!why.empty()) return PSLR_ERR_ARG;
    if (n == 0) return PSLR_OK;
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_dg = nullptr, *d_rows = nullptr, *d_lptr = nullptr,
            *d_blev = nullptr;
    int *d_bad = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int bad = INT_MAX;
    cudaError_t e = upload(d_rp, rp, (size_t)n + 1, st);
    if (e == cudaSuccess) e = upload(d_ci, ci, (size_t)rp[n], st);
    if (e == cudaSuccess) e = upload(d_dg, dg, st);
    if (e == cudaSuccess) e = upload(d_rows, rows, st);
    if (e == cudaSuccess) e = upload(d_lptr, lptr, st);
    if (e == cudaSuccess) e = upload(d_blev, blev, st);
    if (e == cudaSuccess) e = upload(d_bad, std::vector<int>(1, INT_MAX), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        Ilu0Params P{d_rp, d_ci, d_dg, val_dev, d_rows, d_lptr, d_blev, nb, d_bad};
        const int grid = std::max(1, std::min(nb, 65535));
        cudaEventRecord(e0, st);
        k_ilu0_levels<<<grid, kIluThreads, 0, st>>>(P);
        e = cudaGetLastError();
        cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && kernel_ms) cudaEventElapsedTime(kernel_ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_rp);
    cudaFree(d_ci);
    cudaFree(d_dg);
    cudaFree(d_rows);
    cudaFree(d_lptr);
    cudaFree(d_blev);
    cudaFree(d_bad);
    if (e != cudaSuccess) {
        why = std::string("CUDA: ") + cudaGetErrorString(e);
        return PSLR_ERR_CUDA;
    }
    if (bad != INT_MAX) {
        if (bad_row) *bad_row = bad;
        why = "ILU(0) met a zero pivot in row " + std::to_string(bad);
        return PSLR_ERR_ZERO_PIVOT;
    }
    return PSLR_OK;
}

}  // namespace pslr

extern "C" pslr_status pslr_ilu0_device(int32_t n, int32_t nb, const int32_t *block_ptr, const int32_t *rowptr,
                                        const int32_t *colind, double *val_dev, void *stream) {
    if (n < 0 || nb < 0 || !block_ptr || !rowptr || (n > 0 && (nb == 0 || !colind || !val_dev)))
        return PSLR_ERR_ARG;
    std::string why;
    const pslr_status st = pslr::ilu0_device_blocks(n, nb, block_ptr, rowptr, colind, val_dev,
                                                    (cudaStream_t)stream, nullptr, nullptr, why);
    if (st != PSLR_OK) fprintf(stderr, "pslr_ilu0_device: %s\n", why.c_str());
    return st;
}
