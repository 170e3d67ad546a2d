// Graph partition for matrices without a grid: recursive bisection by
// breadth-first level structures, standing in for the METIS partition the
// paper uses (Section 2) when no geometric split applies.
//
// The graph is the pattern of A + A^T without self loops, each vertex's
// neighbours visited in increasing index.  A vertex set U (ascending) is cut
// into k parts as follows.  k = 1: U is one part.  Otherwise U is ordered
// breadth-first: its components are taken in the order of their smallest
// vertex, each searched from a pseudo-peripheral vertex found by the George-Liu
// iteration (start at the component's smallest vertex; search; among the
// vertices of the last level take one of least degree within U, the smallest
// on ties; repeat from it while the number of levels grows).  With k1 = k / 2
// the first floor(|U| k1 / k) vertices of that order form U1, the rest U2
// (both re-sorted ascending); U1 is cut into k1 parts numbered from the base,
// U2 into k - k1 parts numbered after them.  Every step is deterministic, so
// the result depends only on the pattern and k.  The two sides of a cut
// touch disjoint vertices, so the upper levels of the recursion run on host
// threads; the markers the searches share are relaxed atomics, and every
// search compares them only against tags and stamps unique to itself, so the
// result does not depend on the threads either.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

namespace pslr_part {

namespace {

struct Graph {
    std::vector<int32_t> rp, ci;  // symmetric pattern, no self loops, ascending
};

Graph symmetric_pattern(int n, const int32_t *rowptr, const int32_t *colind) {
    std::vector<int32_t> deg(n + 1, 0);
    for (int v = 0; v < n; ++v)
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            const int w = colind[k];
            if (w == v) continue;
            deg[v + 1]++;
            deg[w + 1]++;
        }
    for (int v = 0; v < n; ++v) deg[v + 1] += deg[v];
    std::vector<int32_t> tmp(deg[n]), pos(deg.begin(), deg.end() - 1);
    for (int v = 0; v < n; ++v)
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            const int w = colind[k];
            if (w == v) continue;
            tmp[pos[v]++] = w;
            tmp[pos[w]++] = v;
        }
    Graph g;
    g.rp.assign(1, 0);
    g.ci.reserve(tmp.size());
    for (int v = 0; v < n; ++v) {  // sort and drop duplicates (entries of both a_vw and a_wv)
        auto b = tmp.begin() + deg[v], e = tmp.begin() + deg[v + 1];
        std::sort(b, e);
        auto last = std::unique(b, e);
        g.ci.insert(g.ci.end(), b, last);
        g.rp.push_back((int32_t)g.ci.size());
    }
    return g;
}

class Bisector {
  public:
    Bisector(const Graph &g, int n, int32_t *part)
        : g_(g), part_(part), inset_(new std::atomic<int>[n]), seen_(new std::atomic<int>[n]) {
        for (int v = 0; v < n; ++v) {
            inset_[v].store(0, std::memory_order_relaxed);
            seen_[v].store(0, std::memory_order_relaxed);
        }
    }

    // Cut U into k parts numbered from base; `threads` host threads may share
    // the work below this cut.
    void cut(std::vector<int32_t> &U, int k, int base, int threads) {
        if (k == 1) {
            for (int v : U) part_[v] = base;
            return;
        }
        const int tag = tags_.fetch_add(1) + 1;
        for (int v : U) set(inset_, v, tag);
        std::vector<int32_t> order;
        order.reserve(U.size());
        const int done = stamps_.fetch_add(1) + 1;  // vertices already placed in `order`
        std::vector<int32_t> seq;
        for (int c : U) {
            if (get(seen_, c) == done) continue;
            peripheral(c, tag, done, seq);  // the search from the vertex it picks
            for (int v : seq) set(seen_, v, done);
            order.insert(order.end(), seq.begin(), seq.end());
        }
        const int k1 = k / 2;
        const size_t n1 = (size_t)(((int64_t)U.size() * k1) / k);
        std::vector<int32_t> U1(order.begin(), order.begin() + n1), U2(order.begin() + n1, order.end());
        std::vector<int32_t>().swap(order);
        std::vector<int32_t>().swap(U);
        std::sort(U1.begin(), U1.end());
        std::sort(U2.begin(), U2.end());
        std::thread side;
        if (threads > 1) {
            const int t1 = threads / 2;
            try {
                side = std::thread([&, t1]() {
                    try {
                        cut(U1, k1, base, t1);
                    } catch (...) {
                        failed_ = true;
                    }
                });
            } catch (...) {  // no thread to be had: the same work on this one
            }
        }
        try {
            if (!side.joinable()) cut(U1, k1, base, 1);
            cut(U2, k - k1, base + k1, side.joinable() ? threads - threads / 2 : 1);
        } catch (...) {
            failed_ = true;
        }
        if (side.joinable()) side.join();
    }

    bool failed() const { return failed_; }

  private:
    static int get(const std::unique_ptr<std::atomic<int>[]> &a, int v) {
        return a[v].load(std::memory_order_relaxed);
    }
    static void set(std::unique_ptr<std::atomic<int>[]> &a, int v, int x) {
        a[v].store(x, std::memory_order_relaxed);
    }

    // Breadth-first search from root over the vertices of the set `tag` not
    // marked `done`, under a fresh private stamp; q receives the vertices in
    // the order they are reached.  Returns the number of levels and the index
    // in q where the last level begins.
    int bfs(int root, int tag, int done, std::vector<int32_t> &q, size_t &last_begin) {
        const int mark = stamps_.fetch_add(1) + 1;
        q.clear();
        size_t head = 0;
        set(seen_, root, mark);
        q.push_back(root);
        int levels = 0;
        size_t level_begin = head;
        while (head < q.size()) {
            const size_t level_end = q.size();
            ++levels;
            level_begin = head;
            for (; head < level_end; ++head) {
                const int v = q[head];
                for (int t = g_.rp[v]; t < g_.rp[v + 1]; ++t) {
                    const int w = g_.ci[t];
                    if (get(inset_, w) != tag) continue;
                    const int sw = get(seen_, w);
                    if (sw == mark || sw == done) continue;
                    set(seen_, w, mark);
                    q.push_back(w);
                }
            }
        }
        last_begin = level_begin;
        return levels;
    }

    int degree(int v, int tag) const {
        int d = 0;
        for (int t = g_.rp[v]; t < g_.rp[v + 1]; ++t) d += get(inset_, g_.ci[t]) == tag;
        return d;
    }

    // George-Liu pseudo-peripheral vertex of the component of c; seq
    // receives the breadth-first search from it.
    void peripheral(int c, int tag, int done, std::vector<int32_t> &seq) {
        size_t lb = 0, lbx = 0;
        int ecc = bfs(c, tag, done, seq, lb);
        std::vector<int32_t> sx;
        for (;;) {
            int x = -1, dx = 0;
            for (size_t t = lb; t < seq.size(); ++t) {
                const int v = seq[t];
                const int d = degree(v, tag);
                if (x < 0 || d < dx || (d == dx && v < x)) {
                    x = v;
                    dx = d;
                }
            }
            const int ex = bfs(x, tag, done, sx, lbx);
            if (ex <= ecc) return;
            ecc = ex;
            seq.swap(sx);
            lb = lbx;
        }
    }

    const Graph &g_;
    int32_t *part_;
    std::unique_ptr<std::atomic<int>[]> inset_, seen_;
    std::atomic<int> tags_{0}, stamps_{0};
    std::atomic<bool> failed_{false};
};

}  // namespace

// part[v] in 0..nparts-1 for every vertex; 1 <= nparts <= n; up to
// `threads` host threads.  false if the host ran out of memory.
bool graph_partition(int n, const int32_t *rowptr, const int32_t *colind, int nparts, int32_t *part,
                     int threads) {
    try {
        Graph g = symmetric_pattern(n, rowptr, colind);
        std::vector<int32_t> U(n);
        for (int v = 0; v < n; ++v) U[v] = v;
        Bisector b(g, n, part);
        b.cut(U, nparts, 0, std::max(1, threads));
        return !b.failed();
    } catch (...) {
        return false;
    }
}

}  // namespace pslr_part
