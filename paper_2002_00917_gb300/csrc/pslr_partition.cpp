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
// the result depends only on the pattern and k.
#include <algorithm>
#include <cstdint>
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
    Bisector(const Graph &g, int n, int32_t *part) : g_(g), part_(part), inset_(n, 0), seen_(n, 0) {}

    void cut(std::vector<int32_t> &U, int k, int base) {
        if (k == 1) {
            for (int v : U) part_[v] = base;
            return;
        }
        const int tag = ++tags_;
        for (int v : U) inset_[v] = tag;
        std::vector<int32_t> order;
        order.reserve(U.size());
        const int done = ++stamps_;  // vertices already placed in `order`
        for (int c : U) {
            if (seen_[c] == done) continue;
            const int root = peripheral(c, tag, done);
            bfs(root, tag, done, &order, nullptr);
        }
        const int k1 = k / 2;
        const size_t n1 = (size_t)(((int64_t)U.size() * k1) / k);
        std::vector<int32_t> U1(order.begin(), order.begin() + n1), U2(order.begin() + n1, order.end());
        std::vector<int32_t>().swap(order);
        std::vector<int32_t>().swap(U);
        std::sort(U1.begin(), U1.end());
        std::sort(U2.begin(), U2.end());
        cut(U1, k1, base);
        cut(U2, k - k1, base + k1);
    }

  private:
    // Breadth-first search from root over vertices of the set `tag` that are
    // not marked `done`.  With `out`, every reached vertex is appended to it and
    // marked `done`; otherwise the search uses a fresh private stamp.  Returns
    // the number of levels; `last` (optional) receives the last level.
    int bfs(int root, int tag, int done, std::vector<int32_t> *out, std::vector<int32_t> *last) {
        const int mark = out ? done : ++stamps_;
        std::vector<int32_t> local;
        std::vector<int32_t> &q = out ? *out : local;
        size_t head = q.size();
        seen_[root] = mark;
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
                    if (inset_[w] != tag || seen_[w] == mark || seen_[w] == done) continue;
                    seen_[w] = mark;
                    q.push_back(w);
                }
            }
        }
        if (last) last->assign(q.begin() + level_begin, q.end());
        return levels;
    }

    int degree(int v, int tag) const {
        int d = 0;
        for (int t = g_.rp[v]; t < g_.rp[v + 1]; ++t) d += inset_[g_.ci[t]] == tag;
        return d;
    }

    // George-Liu pseudo-peripheral vertex of the component of c.
    int peripheral(int c, int tag, int done) {
        int r = c;
        std::vector<int32_t> last;
        int ecc = bfs(r, tag, done, nullptr, &last);
        for (;;) {
            int x = -1, dx = 0;
            for (int v : last) {
                const int d = degree(v, tag);
                if (x < 0 || d < dx || (d == dx && v < x)) {
                    x = v;
                    dx = d;
                }
            }
            std::vector<int32_t> lx;
            const int ex = bfs(x, tag, done, nullptr, &lx);
            if (ex <= ecc) return r;
            r = x;
            ecc = ex;
            last.swap(lx);
        }
    }

    const Graph &g_;
    int32_t *part_;
    std::vector<int> inset_, seen_;
    int tags_ = 0, stamps_ = 0;
};

}  // namespace

// part[v] in 0..nparts-1 for every vertex; 1 <= nparts <= n.
void graph_partition(int n, const int32_t *rowptr, const int32_t *colind, int nparts, int32_t *part) {
    Graph g = symmetric_pattern(n, rowptr, colind);
    std::vector<int32_t> U(n);
    for (int v = 0; v < n; ++v) U[v] = v;
    Bisector(g, n, part).cut(U, nparts, 0);
}

}  // namespace pslr_part
