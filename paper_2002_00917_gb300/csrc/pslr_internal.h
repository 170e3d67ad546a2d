// Internal layout shared by the host set-up (pslr_host.cpp) and the kernels.
//
// Device data layout.  Every sparse piece the apply touches - one level of a
// triangular factor, or a slice of the E_i / F_i / C_g,i block of one
// subdomain - is a "segment": a contiguous, 16-byte aligned byte range of
// at most kSegMaxRows rows (one consumer thread per row) that starts with a
// 16-byte SegHdr.  Rows are padded to np = round_up(n, 8).  Two encodings:
//
//   record (fmt kRec3 / kRec7, rows with at most 3 / 7 entries): per row one
//     index record and one value record, so a thread fetches its row with one
//     or two vector loads at j * size and no address arithmetic:
//       idx[np]:  {row, c_0 .. c_{K-1}}   (uint16, or int32 for global columns)
//       val[np]:  {v_0 .. v_{K-1}, dinv}  (value type; dinv = 1/diagonal, or 1)
//     with K = 3 or 7 entries; unused entries point at the zero slot with
//     value 0, so every row runs the same K fused multiply-adds.
//   tile (fmt kTile, wider rows): ELL slot-major,
//       vals[w][np], dinv[np] (with a diagonal), cols[w][np], rows[np].
//
// The zero slot is index n_local of the shared-memory vector (or q for the
// global interface vector), which always holds 0.
//
// A triangular sweep's segment may hold several consecutive levels: blocks of
// the form above, one after the other, every block but the last flagged
// kSegMore, each with its own header and byte size.  Each block is one
// barrier step of the sweep; the segment is one ring slot and one bulk copy.
// Copying a segment costs the producer about as long as a level step, so
// packing levels together (up to kSegBudget bytes) keeps it ahead.
//
// For every launch the host lays out, per CTA, the exact sequence of segments
// its consumers will use (the "stream").  A producer warp walks the stream and
// copies each segment into a shared-memory ring with a TMA bulk copy as soon
// as a slot frees up; consumers take segments from the ring in the same order.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define PSLR_HD __host__ __device__
#else
#define PSLR_HD
#endif

namespace pslr {

constexpr int kConsumers = 256;             // consumer threads (8 warps)
constexpr int kThreads = kConsumers + 32;   // + one producer warp
constexpr int kSegMaxRows = kConsumers;     // rows per segment
constexpr int kSegBudget = 12 * 1024;       // bytes per segment (one ring slot at most)
constexpr int kMaxRing = 32;                // ring slots at most
constexpr int kMinDualRing = 3;             // ring slots at least when two CTAs share an SM
constexpr int kMergeBelowSlots = 6;         // merge sweep levels when a two-CTA ring holds fewer slots
constexpr int kMaxRank = 128;               // largest low-rank term

enum SegFlags : uint32_t { kSegDiag = 1u, kSegGlobalCols = 2u, kSegMore = 4u };
enum SegFmt : uint8_t { kTile = 0, kRec3 = 3, kRec7 = 7 };

struct SegHdr {
    uint16_t n;      // rows
    uint8_t w;       // entries per row (tile: padded width; record: K)
    uint8_t flags;   // SegFlags
    uint16_t np;     // padded rows
    uint8_t fmt;     // SegFmt
    uint8_t pad0;
    uint32_t bytes;  // byte size of this block
    uint32_t pad2;
};
static_assert(sizeof(SegHdr) == 16, "SegHdr is 16 bytes");

// One entry of a CTA's segment stream.
struct StreamEnt {
    int64_t off;     // byte offset of the segment from the segment base
    int32_t bytes;   // byte size (multiple of 16)
    int32_t pad;
};
static_assert(sizeof(StreamEnt) == 16, "StreamEnt is 16 bytes");

PSLR_HD inline int seg_npad(int n) { return (n + 7) & ~7; }

// Record sizes of the kRec3 / kRec7 encodings.
template <class IDX>
PSLR_HD inline int rec_idx_bytes(int K) {
    return (K + 1) * (int)sizeof(IDX);
}
template <class T>
PSLR_HD inline int rec_val_bytes(int K) {
    return (K + 1) * (int)sizeof(T);
}

// Bytes of a segment of n rows and width w (fmt chosen from w).
PSLR_HD inline int seg_fmt_for(int w) { return w <= 3 ? kRec3 : (w <= 7 ? kRec7 : kTile); }

template <class T, class IDX>
PSLR_HD inline int64_t seg_bytes(int n, int w, bool diag) {
    const int64_t np = seg_npad(n);
    const int fmt = seg_fmt_for(w);
    if (fmt != kTile) return 16 + np * (rec_idx_bytes<IDX>(fmt) + rec_val_bytes<T>(fmt));
    return 16 + np * w * (int64_t)sizeof(T) + (diag ? np * (int64_t)sizeof(T) : 0) +
           np * w * (int64_t)sizeof(IDX) + np * 2;
}

// Segment counts of one subdomain, in stream order of its descriptor table:
// E, F, C_g, sweep 1 of the B solve, sweep 2 of the B solve, sweep 1 and
// sweep 2 of the C0 solve.  In the forward direction the B solve is L then U
// and E, F, C_g are E_i, F_i and the rows of C_g of subdomain i; in the
// transposed direction the solve is U^T then L^T and the slots hold F_i^T,
// E_i^T and the rows of C_g^T of subdomain i.
enum { kE = 0, kF = 1, kCg = 2, kB1 = 3, kB2 = 4, kC1 = 5, kC2 = 6, kNCnt = 7 };

// Parameters of one launch of the persistent apply kernel: arithmetic in T,
// the caller's vectors b and z in IO (IO = double with T = float is the FP32
// preconditioner applied to FP64 Krylov vectors, converting on the fly).
template <class T, class IO = T>
struct ApplyParams {
    const char *segbase;         // segments of this direction and precision
    const StreamEnt *stream;     // all CTAs' streams
    const int64_t *stream_off;   // grid+1: CTA b uses stream[stream_off[b] .. stream_off[b+1])
    const int32_t *cnt;          // kNCnt*s segment counts
    int ring, slot_bytes;        // ring slots and slot size
    int pivot_post;              // exact LU: 0 gather rhs before the sweeps, 1 scatter after
    int lowrank_after;           // 0: t <- t + V G V^T t before the series (Algorithm 3)
                                 // 1: w <- w + V G^T V^T w after it (transpose)
    int s, p, q, r, m, grid;
    int max_p, max_q;            // shared-memory sizing
    const int32_t *ioff, *goff;  // s+1 interior / interface offsets
    const int32_t *perm;         // n: reordered index -> original index
    const uint16_t *bpiv;        // p: exact-LU row permutation of B (local), or nullptr
    const uint16_t *cpiv;        // q: exact-LU row permutation of C0 (local), or nullptr
    const void *V;               // q x r row-major, row stride ldv: double (FP64) or bf16 (FP32)
    int ldv;                     // row stride of V: r rounded up to a multiple of 8 (zero padded)
    const T *G;                  // r x r column-major (G, or G^T for the transpose)
    const IO *b;                 // n input, original order
    IO *z;                       // n output, original order
    T *wbuf;                     // 2*(q+1): series iterates (ping-pong; slot q stays 0)
    T *acc;                      // q: series accumulator / low-rank staging
    T *part;                     // s*r: per-subdomain partial V^T t
    unsigned *bar;               // [0] arrivals, [1] generation
    int *err;                    // latched error (pslr_status)
    const int *skip;             // when *skip != 0 the launch does nothing (converged FGMRES cycle)
    long long wait_limit;        // polls before a grid-barrier wait gives up
    int rs;                      // column stride of the low-rank reduction scratch (red_stride(r))
    T omega;                     // series scaling: 1 for PSLR (Eq. 3.3); otherwise the Sec. 1
                                 // Neumann polynomial, w_k = (1-omega) w_{k-1} + omega C0^{-1} E_s w_{k-1},
                                 // y = omega sum w_k (no low-rank term)
    const T *dB, *dC;            // unit-diagonal form (the kernels' kUnit instances): p and q inverse
                                 // diagonals of the U factors of B_i and C0_i, reordered order, by
                                 // which every sweep's right-hand side is scaled; nullptr otherwise
};

// E_rr(m) v for the Arnoldi process (Eq. 3.19): v <- (E_s C0^{-1})^{m+1} v.
template <class T>
struct ErrParams {
    const char *segbase;
    const StreamEnt *stream;
    const int64_t *stream_off;
    const int32_t *cnt;
    int ring, slot_bytes;
    int s, p, q, m, grid;
    int max_p, max_q;
    const int32_t *ioff, *goff;
    const uint16_t *bpiv, *cpiv;
    const T *vin;                // q (interface numbering)
    T *vout;                     // q: carried iterate between repetitions, then the result
    T *abuf;                     // 2*(q+1): C0^{-1} v per repetition, ping-pong (slot q = 0)
    unsigned *bar;
    int *err;
    long long wait_limit;
    int rs;                      // as in ApplyParams (the layout must match the apply's)
};

// Batched apply (pslr_batch.cuh): per-system parameters and launch parameters.
constexpr int kMaxBatchRhs = 4;             // right-hand sides per system in one batched launch
constexpr int kMaxGroup = 8;                // subdomains of one system swept in lockstep by one CTA

// A group: up to kMaxGroup subdomains of one system that one CTA sweeps in
// lockstep.  Their local vectors are concatenated in shared memory (item t's
// interior part at xo[t] .. xo[t] + p_i, its zero slot last; likewise the
// interface part at go[t]), and the group's merged segments index those
// concatenated vectors: merged level j holds level j of every item.
struct BatchGroup {
    int32_t sys, n;                 // system, items (1..kMaxGroup)
    int32_t sub[kMaxGroup];         // subdomain of each item
    int32_t xo[kMaxGroup + 1];      // interior offsets (item t spans p_i + 1 entries)
    int32_t go[kMaxGroup + 1];      // interface offsets (item t spans q_i + 1 entries)
    int32_t cnt[kNCnt];             // merged segments per category
};

template <class T>
struct BatchSys {
    const int32_t *ioff, *goff, *perm;
    const void *V;              // q x r row-major, row stride ldv: double (FP64) or bf16 (FP32)
    const T *G;                 // r x r column-major
    T *wbuf;                    // nrhs blocks of 2(q+1): series iterates (ping-pong, slot q = 0)
    T *acc;                     // nrhs blocks of q+1: accumulator
    T *part;                    // nrhs blocks of s*r: per-subdomain partials of V^T t
    T *dco;                     // nrhs blocks of r: low-rank coefficients d = G V^T t
    int64_t voff;               // start of the system's n x nrhs block in b and z
    int n, s, p, q, r, m;
    int ldv;                    // row stride of V (r rounded up to a multiple of 8)
};

template <class T, class IO>
struct BatchParams {
    const BatchSys<T> *sys;
    const char *segbase;        // the batch's merged segments (stream offsets are relative to it)
    const BatchGroup *groups;   // grouped by CTA
    const int32_t *group_off;   // grid+1
    const int32_t *pairs;       // (system, rhs) pairs of systems with r > 0, grouped by CTA
    const int32_t *pair_off;    // grid+1
    const StreamEnt *stream;
    const int64_t *stream_off;  // grid+1
    const IO *b;                // batched input (system-major, n_k x nrhs column-major per system)
    IO *z;                      // batched output, same layout
    int ring, slot_bytes;
    int xs, gs;                 // per-rhs strides of a group's interior / interface vectors in shared memory
    int max_m, nrhs, grid, any_lr;
    int pair64;                 // FP64, nrhs > 1: one thread per (row, rhs) pair (else one per row)
    unsigned *bar;
    int *err;
    const int *skip;            // when *skip != 0 the launch does nothing
    const int *active;          // nsys flags, or nullptr: systems with active[k] == 0 are skipped
    long long wait_limit;
};

// Batched FGMRES (pslr_bkrylov.cu).  A "problem" is one (system, right-hand
// side) pair: a contiguous range of the batched vector.  Each problem is cut
// into chunks of at most kBkChunk rows; one CTA handles one chunk, and every
// per-problem reduction adds its chunks' partials in chunk order.  Small
// chunks keep every SM's FP64 pipe busy once only a few problems still run
// (64-system batched FGMRES(127): 3.08 s with 4096 rows, 2.87 s with 2048,
// 2.85 s with 1024 in the FP32 form).
constexpr int kBkChunk = 1024;

struct BkProb {
    int64_t off;        // first element of the problem in the batched vector
    int32_t n, sys;     // length, system
    int32_t c0, nc;     // its chunks
};

struct BkChunk {
    int64_t b, e;       // element range in the batched vector
    int32_t prob, pad;
};

struct BkSys {          // the system's matrix A (CSR, original ordering)
    const int32_t *rp, *ci;
    const double *av;
};

// Per-problem FGMRES state (device arrays of length nprob unless noted).
struct BkState {
    int *stop;          // no further Arnoldi steps in this cycle
    int *jd;            // Arnoldi steps done in this cycle
    int *conv;          // 0 running, 1 converged, 2 stopped (maxit), 3 not finite
    int *its;           // iterations so far
    double *bn, *rn, *hn, *relres;
    double *H;          // nprob x (K+1) x K, column-major per problem
    double *rot;        // nprob x 2K: cosines then sines
    double *gam;        // nprob x (K+1)
    double *h1, *h2;    // nprob x (K+1): the two CGS coefficient vectors of this step
    double *y;          // nprob x K: least-squares solution of the cycle
    double *pa, *pb;    // nchunk x (K+1): per-chunk partials (ping-pong)
    int *remaining;     // [1] problems still running
    int *skip;          // [1] no problem running: later launches of the cycle return at once
    int *sys_active;    // nsys: some problem of the system still runs (the apply skips the others)
    int nsys, nrhs;     // problem p belongs to system p / nrhs
    const double *rtol;  // [1] device: relative tolerance of this solve
    const int *maxit;    // [1] device: iteration limit of this solve (both outside the cycle graph)
    int K;              // restart length
};

// Shared-memory layout of the persistent kernels (host and device agree on it).
struct SmemLayout {
    int ring, full, empty, ctl, xi, wi, si, tmp, red, total;
};

PSLR_HD inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Low-rank reduction scratch (8-byte entries) for a column stride rs >= rank:
// 8 warps' partial sums of rs columns (or the kConsumers group sums of
// lowrank_coeffs, whichever is larger), then u and d of rs entries each.
PSLR_HD inline int red_u_off(int rs) { return 8 * rs > kConsumers ? 8 * rs : kConsumers; }
PSLR_HD inline int red_bytes(int rs) { return align_up((red_u_off(rs) + 2 * rs) * 8, 128); }

// Column stride of the reduction scratch for a rank r (kMaxRank for the
// batched kernel, whose ranks differ per system).
PSLR_HD inline int red_stride(int r) { return r < 8 ? 8 : (r + 7) / 8 * 8; }

// alias_w: the interface vectors wi and si share one buffer.  The
// single-system apply and E_rr kernels never hold both at once (wi only feeds
// the E product that starts a series term, or the last phase, where si is
// unused); the batched kernel does, and keeps them apart.
PSLR_HD inline int smem_fixed(int max_p, int max_q, int tsize, bool pivots, int rs = kMaxRank,
                              bool alias_w = false) {
    int o = 2 * align_up(kMaxRing * 8, 16) + 128;
    o = align_up(o, 128);
    o += align_up((max_p + 1) * tsize, 128);
    o += (alias_w ? 1 : 2) * align_up((max_q + 1) * tsize, 128);
    o += pivots ? align_up(((max_p > max_q ? max_p : max_q) + 1) * tsize, 128) : 0;
    o += red_bytes(rs);
    return o;
}

PSLR_HD inline SmemLayout smem_layout(int slot_bytes, int ring, int max_p, int max_q, int tsize,
                                      bool pivots, int rs = kMaxRank, bool alias_w = false) {
    SmemLayout L;
    int o = 0;
    L.ring = o;  o += ring * slot_bytes;
    L.full = o;  o += align_up(kMaxRing * 8, 16);
    L.empty = o; o += align_up(kMaxRing * 8, 16);
    L.ctl = o;   o += 128;
    o = align_up(o, 128);
    L.xi = o;    o += align_up((max_p + 1) * tsize, 128);
    L.wi = o;    o += alias_w ? 0 : align_up((max_q + 1) * tsize, 128);
    L.si = o;    o += align_up((max_q + 1) * tsize, 128);
    L.tmp = o;   o += pivots ? align_up(((max_p > max_q ? max_p : max_q) + 1) * tsize, 128) : 0;
    L.red = o;   o += red_bytes(rs);
    L.total = o;
    return L;
}

}  // namespace pslr
