// Internal layout shared by the host set-up (pslr_host.cpp) and the kernels.
//
// Device data layout.  Every sparse piece the apply touches - one level of a
// triangular factor, or the E_i / F_i / C_g,i block of one subdomain - is a
// "segment": a contiguous, 16-byte aligned byte range holding an ELL tile
// (rows padded to npad = round_up(n, 8), entries slot-major):
//
//     val_t vals[w][npad];   val_t dinv[npad] (only with a diagonal);
//     idx_t cols[w][npad];   uint16 rows[npad];
//
// idx_t is uint16 for subdomain-local columns and int32 for the global
// interface columns of C_g.  Padded entries point at a zero slot (local index
// n_local, or q for the global interface vector) with value 0.  Segments are
// staged into shared memory by TMA bulk copies (cp.async.bulk) a few ahead of
// their use, so the dependent chain of a triangular solve never waits on L2.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define PSLR_HD __host__ __device__
#else
#define PSLR_HD
#endif

namespace pslr {

constexpr int kThreads = 256;      // threads per CTA of the persistent kernels
constexpr int kRing = 4;           // segments in flight per CTA
constexpr int kMaxRank = 64;       // largest low-rank term

enum SegFlags : uint32_t { kSegDiag = 1u, kSegGlobalCols = 2u };

struct SegDesc {
    int64_t off;     // byte offset from the segment base (multiple of 16)
    int32_t bytes;   // byte size (multiple of 16); 0 = empty segment
    uint16_t n;      // rows
    uint8_t w;       // entries per row after padding
    uint8_t flags;   // SegFlags
};
static_assert(sizeof(SegDesc) == 16, "SegDesc is 16 bytes");

PSLR_HD inline int seg_npad(int n) { return (n + 7) & ~7; }

template <class T, class IDX>
PSLR_HD inline int64_t seg_bytes(int n, int w, bool diag) {
    int64_t np = seg_npad(n);
    return np * w * (int64_t)sizeof(T) + (diag ? np * (int64_t)sizeof(T) : 0) +
           np * w * (int64_t)sizeof(IDX) + np * 2;
}

// Per-subdomain descriptor table, in this order: the segments of E, of F, of
// C_g, of sweep 1 of the B solve, of sweep 2 of the B solve, of sweep 1 of
// the C0 solve and of sweep 2 of the C0 solve (cnt[7] per subdomain gives the
// number of each).  A level or block larger than kSegBudget bytes is split
// into several segments.  In the forward direction the B solve is L then U
// and E, F, C_g are E_i, F_i and the rows of C_g of subdomain i; in the
// transposed direction the solve is U^T then L^T and the slots hold F_i^T,
// E_i^T and the rows of C_g^T of subdomain i.
enum { kE = 0, kF = 1, kCg = 2, kB1 = 3, kB2 = 4, kC1 = 5, kC2 = 6, kNCnt = 7 };
constexpr int kSegBudget = 12 * 1024;  // bytes per segment (one ring slot)
constexpr int kSegMaxRows = 256;       // rows per segment (one per thread)

// Everything one direction (forward or transposed) of one precision needs.
struct OpSetDev {
    const char *segbase;       // all segments of this direction and precision
    const SegDesc *desc;       // descriptor tables of all subdomains
    const int32_t *sub_desc;   // s: first descriptor of subdomain i
    const int32_t *cnt;        // kNCnt*s: segment counts of E, F, Cg, B1, B2, C1, C2
    int pivot_post;            // exact LU: 0 gather rhs before the B/C0 sweeps, 1 scatter after
    int lowrank_after;         // 0: t <- t + V G V^T t before the series (Algorithm 3)
                               // 1: w <- w + V G^T V^T w after it (transpose)
};

// Parameters of one launch of the persistent apply kernel.
template <class T>
struct ApplyParams {
    OpSetDev ops;
    int s, p, q, r, m, grid;
    int max_p, max_q, max_desc;  // shared-memory sizing
    int slot_bytes;              // ring slot size
    const int32_t *ioff, *goff;  // s+1 interior / interface offsets
    const int32_t *perm;         // n: reordered index -> original index
    const uint16_t *bpiv;        // p: exact-LU row permutation of B (local), or nullptr
    const uint16_t *cpiv;        // q: exact-LU row permutation of C0 (local), or nullptr
    const void *V;               // q x r column-major: double (FP64) or bf16 (FP32)
    const T *G;                  // r x r column-major (G, or G^T for the transpose)
    const T *b;                  // n input, original order
    T *z;                        // n output, original order
    T *wbuf;                     // 2*(q+1): series iterates (ping-pong; slot q stays 0)
    T *acc;                      // q: series accumulator / low-rank staging
    T *part;                     // s*r: per-subdomain partial V^T t
    unsigned *bar;               // [0] arrivals, [1] generation
    int *err;                    // latched error (pslr_status)
    const int *skip;             // when *skip != 0 the launch does nothing (converged FGMRES cycle)
    long long wait_limit;        // polls before a wait gives up
};

// E_rr(m) v for the Arnoldi process (Eq. 3.19): v <- (E_s C0^{-1})^{m+1} v.
template <class T>
struct ErrParams {
    OpSetDev ops;                // forward direction
    int s, p, q, m, grid;
    int max_p, max_q, max_desc, slot_bytes;
    const int32_t *ioff, *goff;
    const uint16_t *bpiv, *cpiv;
    const T *vin;                // q (interface numbering)
    T *vout;                     // q: carried iterate between repetitions, then the result
    T *abuf;                     // 2*(q+1): C0^{-1} v per repetition, ping-pong (slot q = 0)
    unsigned *bar;
    int *err;
    long long wait_limit;
};

// Shared-memory layout of the persistent kernels (host and device agree on it).
struct SmemLayout {
    int ring, mbar, desc, xi, wi, si, tmp, red, total;
};

PSLR_HD inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

PSLR_HD inline SmemLayout smem_layout(int slot_bytes, int max_desc, int max_p,
                                                  int max_q, int tsize, bool pivots) {
    SmemLayout L;
    int o = 0;
    L.ring = o;  o += kRing * slot_bytes;
    L.mbar = o;  o += align_up(kRing * 8, 128);
    L.desc = o;  o += align_up(max_desc * 16, 128);
    L.xi = o;    o += align_up((max_p + 1) * tsize, 128);
    L.wi = o;    o += align_up((max_q + 1) * tsize, 128);
    L.si = o;    o += align_up((max_q + 1) * tsize, 128);
    L.tmp = o;   o += pivots ? align_up(((max_p > max_q ? max_p : max_q) + 1) * tsize, 128) : 0;
    L.red = o;   o += align_up((kThreads / 32 + 2) * kMaxRank * 8, 128);
    L.total = o;
    return L;
}

}  // namespace pslr
