/*
 * CPU oracle for list ranking and connected components.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls this code: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg and reference
 * arm load it.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Both problems have exact, unique answers, so the oracle computes the plain
 * definitions sequentially and does not follow the parallel algorithms:
 *
 *  - List ranking (Sec. 3): a linked list is given as a successor array; the
 *    rank of an element is its distance to the last element of the list. The
 *    oracle walks the list once from its head and numbers the elements.
 *  - Weighted list ranking (Sec. 3.2, the sublist value sum in place of the
 *    length): the sum of per-element values from an element to its tail, for
 *    one list or for every list of a forest (heads found by in-degree).
 *  - Connected components (Sec. 4): for an undirected graph given as an edge
 *    list, two vertices share a label iff they are joined by a path. The label
 *    of a component is its smallest vertex id. Two independent computations
 *    are given: breadth-first search started from every unvisited vertex in
 *    increasing id order, and union-find.
 *
 * Conventions. Node ids are int32. A tail is an element whose successor is -1
 * or the element itself (Sec. 3 marks the last element with succ[j] = j). A
 * valid list input is exactly one list that contains all n elements.
 * Return codes: 0 = OK, 1 = bad argument, 4 = the input is not a single list
 * (or an edge endpoint is out of range).
 *
 * Parity pins: weighted ranks against a reversed cumulative sum over the
 * generator's layout, brute force over small layouts and small forests (whose
 * count is a sum of Lah numbers) and hand-worked fixtures; list ranks are
 * checked against the closed form of the
 * generator's layout, brute force over all small layouts and the invariants
 * rank[tail] = 0, rank[i] = rank[succ[i]] + 1; component labels are checked
 * between the two oracles, against brute force on every graph with five
 * vertices, against graphs with a known number of components and against
 * scipy's connected_components.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ARG 1
#define ORC_INVALID 4

/* ---------------------------------------------------------------- lists -- */

/*
 * Sequential list ranking by one walk from the head (Sec. 3, definition of
 * rank). First pass: rank[cur] receives the walk position k of each element
 * and detects revisits; second pass: rank = n - 1 - k.
 */
int oracle_lr_rank(const int32_t* succ, int64_t n, int32_t head, int32_t* rank) {
    if (n < 0) return ORC_ARG;
    if (n == 0) return ORC_OK;
    if (head < 0 || head >= n) return ORC_ARG;
    for (int64_t i = 0; i < n; ++i) rank[i] = -1;
    int64_t k = 0;
    int64_t cur = head;
    for (;;) {
        if (rank[cur] != -1) return ORC_INVALID;       /* cycle */
        rank[cur] = (int32_t)k;
        int64_t nxt = succ[cur];
        if (nxt == -1 || nxt == cur) break;             /* tail */
        if (nxt < 0 || nxt >= n) return ORC_INVALID;
        cur = nxt;
        ++k;
    }
    if (k + 1 != n) return ORC_INVALID;                 /* not every element is on the list */
    for (int64_t i = 0; i < n; ++i) rank[i] = (int32_t)(n - 1 - rank[i]);
    return ORC_OK;
}

/*
 * Weighted list ranking (the generalisation the paper's Sec. 3.2 notes: the
 * sublist value sum replaces the sublist length): out[i] is the sum of val[j]
 * over the elements j from i to the tail of its list, both included. Sums are
 * taken modulo 2^32 (unsigned arithmetic, stored as int32), which is exact
 * whenever the true sums fit in an int32. With val = 1 everywhere, out = rank + 1.
 *
 * One list with a given head: one walk from the head records the order, then
 * the sums are accumulated from the tail back to the head.
 */
int oracle_lr_scan(const int32_t* succ, const int32_t* val, int64_t n, int32_t head, int32_t* out) {
    if (n < 0) return ORC_ARG;
    if (n == 0) return ORC_OK;
    if (head < 0 || head >= n) return ORC_ARG;
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!order) return ORC_ARG;
    for (int64_t i = 0; i < n; ++i) out[i] = 0;
    /* out[] doubles as a visited mark during the walk (1 = visited) */
    int64_t k = 0;
    int64_t cur = head;
    int rc = ORC_OK;
    for (;;) {
        if (out[cur]) { rc = ORC_INVALID; break; }        /* cycle */
        out[cur] = 1;
        order[k++] = (int32_t)cur;
        int64_t nxt = succ[cur];
        if (nxt == -1 || nxt == cur) break;                /* tail */
        if (nxt < 0 || nxt >= n) { rc = ORC_INVALID; break; }
        cur = nxt;
    }
    if (rc == ORC_OK && k != n) rc = ORC_INVALID;          /* not every element is on the list */
    if (rc == ORC_OK) {
        uint32_t acc = 0;
        for (int64_t j = n - 1; j >= 0; --j) {
            acc += (uint32_t)val[order[j]];
            out[order[j]] = (int32_t)acc;
        }
    }
    free(order);
    return rc;
}

/*
 * Weighted list ranking of a forest of lists (every element belongs to
 * exactly one list; no head is given). An in-degree count finds the heads
 * (elements that no successor names); any element named twice, or elements
 * left over after walking every list from its head (a cycle), make the input
 * invalid. Each list is then summed as in oracle_lr_scan.
 */
int oracle_lr_scan_forest(const int32_t* succ, const int32_t* val, int64_t n, int32_t* out) {
    if (n < 0) return ORC_ARG;
    if (n == 0) return ORC_OK;
    int32_t* indeg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!indeg || !order) { free(indeg); free(order); return ORC_ARG; }
    int rc = ORC_OK;
    for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
        int64_t nxt = succ[i];
        if (nxt == -1 || nxt == i) continue;
        if (nxt < 0 || nxt >= n) { rc = ORC_INVALID; break; }
        if (++indeg[nxt] > 1) rc = ORC_INVALID;            /* two predecessors */
    }
    int64_t seen = 0;
    for (int64_t h = 0; h < n && rc == ORC_OK; ++h) {
        if (indeg[h] != 0) continue;                        /* not a head */
        int64_t k = 0;
        int64_t cur = h;
        for (;;) {
            order[k++] = (int32_t)cur;
            int64_t nxt = succ[cur];
            if (nxt == -1 || nxt == cur) break;
            cur = nxt;
        }
        uint32_t acc = 0;
        for (int64_t j = k - 1; j >= 0; --j) {
            acc += (uint32_t)val[order[j]];
            out[order[j]] = (int32_t)acc;
        }
        seen += k;
    }
    if (rc == ORC_OK && seen != n) rc = ORC_INVALID;       /* elements on cycles have no head */
    free(indeg);
    free(order);
    return rc;
}

/*
 * Independent lists, concatenated: list k owns [off[k], off[k+1]) and uses
 * local ids; each is ranked on its own with oracle_lr_rank.
 */
int oracle_lr_rank_batched(const int32_t* succ, const int64_t* off, const int32_t* heads,
                           int64_t count, int32_t* rank) {
    for (int64_t k = 0; k < count; ++k) {
        int64_t b = off[k], e = off[k + 1];
        if (e < b) return ORC_ARG;
        int rc = oracle_lr_rank(succ + b, e - b, heads[k], rank + b);
        if (rc) return rc;
    }
    return ORC_OK;
}

/* ----------------------------------------------------------- components -- */

static int check_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n) {
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_INVALID;
    return ORC_OK;
}

/*
 * Connected components by breadth-first search (Sec. 4, definition of a
 * component). An adjacency array holding both directions of every edge is
 * built by counting; searches start from vertices in increasing id order, so
 * the start vertex is the smallest id of its component and becomes the label.
 */
int oracle_cc_bfs(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label) {
    if (n < 0 || m < 0) return ORC_ARG;
    if (n == 0) return m == 0 ? ORC_OK : ORC_INVALID;
    if (check_edges(src, dst, m, n)) return ORC_INVALID;
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!start || !adj || !queue) { free(start); free(adj); free(queue); return ORC_ARG; }
    for (int64_t e = 0; e < m; ++e) { start[src[e] + 1]++; start[dst[e] + 1]++; }
    for (int64_t v = 0; v < n; ++v) start[v + 1] += start[v];
    int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!fill) { free(start); free(adj); free(queue); return ORC_ARG; }
    memcpy(fill, start, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        adj[fill[src[e]]++] = dst[e];
        adj[fill[dst[e]]++] = src[e];
    }
    free(fill);
    for (int64_t v = 0; v < n; ++v) label[v] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (label[s] != -1) continue;
        int64_t qh = 0, qt = 0;
        label[s] = (int32_t)s;
        queue[qt++] = (int32_t)s;
        while (qh < qt) {
            int32_t u = queue[qh++];
            for (int64_t a = start[u]; a < start[u + 1]; ++a) {
                int32_t w = adj[a];
                if (label[w] == -1) { label[w] = (int32_t)s; queue[qt++] = w; }
            }
        }
    }
    free(start); free(adj); free(queue);
    return ORC_OK;
}

/* Root of x with path halving (every other node on the path skips a level). */
static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/*
 * Connected components by union-find: every edge unites the sets of its
 * endpoints, and the set with the larger root is linked below the smaller
 * root, so each root is the smallest id of its set. The label is the root.
 */
int oracle_cc_uf(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t* label) {
    if (n < 0 || m < 0) return ORC_ARG;
    if (n == 0) return m == 0 ? ORC_OK : ORC_INVALID;
    if (check_edges(src, dst, m, n)) return ORC_INVALID;
    for (int64_t v = 0; v < n; ++v) label[v] = (int32_t)v;
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = uf_find(label, src[e]);
        int32_t b = uf_find(label, dst[e]);
        if (a < b) label[b] = a;
        else if (b < a) label[a] = b;
    }
    for (int64_t v = 0; v < n; ++v) label[v] = uf_find(label, (int32_t)v);
    return ORC_OK;
}

/*
 * Independent graphs, concatenated: graph k owns edges [eoff[k], eoff[k+1])
 * and vertices [voff[k], voff[k+1]), with local ids; labels are local.
 */
int oracle_cc_batched(const int32_t* src, const int32_t* dst, const int64_t* eoff,
                      const int64_t* voff, int64_t count, int32_t* label, int use_uf) {
    for (int64_t k = 0; k < count; ++k) {
        int64_t eb = eoff[k], ee = eoff[k + 1], vb = voff[k], ve = voff[k + 1];
        if (ee < eb || ve < vb) return ORC_ARG;
        int rc = use_uf ? oracle_cc_uf(src + eb, dst + eb, ee - eb, ve - vb, label + vb)
                        : oracle_cc_bfs(src + eb, dst + eb, ee - eb, ve - vb, label + vb);
        if (rc) return rc;
    }
    return ORC_OK;
}
