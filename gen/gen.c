/*
 * Seeded synthetic inputs for list ranking and connected components.
 *
 * This module only creates inputs. It contains none of the arithmetic of the
 * ranking or labelling methods, and both the CPU oracle and the CUDA path are
 * fed from it.
 *
 * Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Output k >= 1 of the stream
 * seeded with s is mix(s + k * GOLDEN), so any element of a stream can be drawn
 * directly from its counter; this makes the parallel generators below
 * independent of the thread count. Unbiased bounded integers use Lemire's
 * multiply-and-reject method ("Fast random integer generation in an interval",
 * ACM TOMACS 2019).
 *
 * Workload shapes follow the paper's experiments: random linked lists stored
 * as successor arrays (Sec. 3, list ranking), uniformly random graphs
 * (Sec. 4, connected components) and R-MAT graphs (Chakrabarti, Zhan &
 * Faloutsos, SDM 2004) for the large skewed case.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* k-th output (k >= 1) of the SplitMix64 stream seeded with s. */
static inline uint64_t sm64_at(uint64_t s, uint64_t k) { return sm64_mix(s + k * GOLDEN); }

/* Sequential stream state. */
typedef struct { uint64_t s; } sm64;
static inline uint64_t sm64_next(sm64* g) { g->s += GOLDEN; return sm64_mix(g->s); }

/* Independent sub-stream seed derived from a seed and a tag. */
static inline uint64_t derive(uint64_t seed, uint64_t tag) {
    return sm64_mix(seed ^ sm64_mix(tag + 0x632be59bd9b4e019ULL));
}

/* Uniform integer in [0, bound) from the sequential stream (Lemire). */
static inline uint64_t sm64_bounded(sm64* g, uint64_t bound) {
    __uint128_t m = (__uint128_t)sm64_next(g) * bound;
    uint64_t l = (uint64_t)m;
    if (l < bound) {
        uint64_t t = (0 - bound) % bound;
        while (l < t) {
            m = (__uint128_t)sm64_next(g) * bound;
            l = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* Multiply-high map of a 64-bit word onto [0, bound). The bias is below
 * bound / 2^64, which is under 2^-32 for every bound used here. */
static inline uint64_t map_bounded(uint64_t x, uint64_t bound) {
    return (uint64_t)(((__uint128_t)x * bound) >> 64);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double to_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Fisher-Yates (Durstenfeld) shuffle of perm[0..n-1] := identity. */
void gen_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    sm64 g = { derive(seed, 1) };
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_bounded(&g, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/*
 * One singly linked list of n nodes in a uniformly random layout: the k-th
 * node of the list is stored at index perm[k]. succ[perm[k]] = perm[k+1],
 * the tail has succ = -1, and *head = perm[0]. perm may be NULL; when it is
 * given it receives the layout, from which the rank of every node is known
 * in closed form (rank[perm[k]] = n-1-k).
 */
int gen_list_random(int64_t n, uint64_t seed, int32_t* succ, int32_t* head, int32_t* perm) {
    if (n <= 0) { if (head) *head = -1; return 0; }
    int32_t* p = perm ? perm : (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!p) return 2;
    gen_permutation(n, seed, p);
    for (int64_t k = 0; k + 1 < n; ++k) succ[p[k]] = p[k + 1];
    succ[p[n - 1]] = -1;
    *head = p[0];
    if (!perm) free(p);
    return 0;
}

/* The ordered control: succ[i] = i+1, tail n-1, head 0. */
void gen_list_ordered(int64_t n, int32_t* succ, int32_t* head) {
    for (int64_t i = 0; i + 1 < n; ++i) succ[i] = (int32_t)(i + 1);
    if (n > 0) succ[n - 1] = -1;
    *head = n > 0 ? 0 : -1;
}

/*
 * Erdos-Renyi style multigraph: m edges with both endpoints drawn uniformly
 * and independently from [0, n). Self-loops and repeated edges are kept.
 * Edge e uses counter e of two independent streams.
 */
void gen_er(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    uint64_t su = derive(seed, 2), sv = derive(seed, 3);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        src[e] = (int32_t)map_bounded(sm64_at(su, (uint64_t)e + 1), (uint64_t)n);
        dst[e] = (int32_t)map_bounded(sm64_at(sv, (uint64_t)e + 1), (uint64_t)n);
    }
}

/*
 * R-MAT graph: n = 2^scale vertices, m edges. Each edge descends scale levels
 * of the adjacency matrix, choosing the quadrant (top-left, top-right,
 * bottom-left, bottom-right) with probabilities (a, b, c, 1-a-b-c). The vertex
 * ids are then relabelled by a seeded random permutation so that the
 * high-degree vertices are spread over the id space.
 */
int gen_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
             int32_t* src, int32_t* dst) {
    if (scale < 0 || scale > 30) return 1;
    int64_t n = (int64_t)1 << scale;
    int32_t* relabel = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!relabel) return 2;
    gen_permutation(n, derive(seed, 4), relabel);
    uint64_t s = derive(seed, 5);
    double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            double x = to_unit(sm64_at(s, (uint64_t)e * (uint64_t)scale + (uint64_t)l + 1));
            uint64_t bu = x >= ab;                       /* bottom half */
            uint64_t bv = (x >= a && x < ab) || x >= abc; /* right half */
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[e] = relabel[u];
        dst[e] = relabel[v];
    }
    free(relabel);
    return 0;
}

/*
 * Instance sizes for a batch: count sizes floor(2^(lo + (hi-lo)*u)) with u
 * uniform in [0, 1), i.e. log-uniform in [2^lo, 2^hi).
 */
void gen_loguniform_sizes(int64_t count, double lo, double hi, uint64_t seed, int64_t* sizes) {
    uint64_t s = derive(seed, 6);
    for (int64_t k = 0; k < count; ++k) {
        double u = to_unit(sm64_at(s, (uint64_t)k + 1));
        int64_t v = (int64_t)floor(pow(2.0, lo + (hi - lo) * u));
        sizes[k] = v < 1 ? 1 : v;
    }
}

/*
 * A batch of independent random lists, concatenated. List k owns nodes
 * [off[k], off[k+1]) of succ; succ values and heads are LOCAL ids (0-based
 * within the list). off must hold count+1 entries and is filled from sizes.
 * perm (may be NULL) receives each list's permutation at the list's own
 * offset, in local ids: list k visits perm[off[k]], perm[off[k] + 1], ...
 */
int gen_list_batch(int64_t count, const int64_t* sizes, uint64_t seed,
                   int64_t* off, int32_t* succ, int32_t* heads, int32_t* perm) {
    off[0] = 0;
    for (int64_t k = 0; k < count; ++k) off[k + 1] = off[k] + sizes[k];
    int rc = 0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(|:rc)
    for (int64_t k = 0; k < count; ++k)
        rc |= gen_list_random(sizes[k], derive(seed, 1000 + (uint64_t)k), succ + off[k], heads + k,
                              perm ? perm + off[k] : NULL);
    return rc;
}

/*
 * A batch of independent uniform random graphs, concatenated. Graph k has
 * vsizes[k] vertices and deg_num * vsizes[k] / deg_den edges; its edges are
 * [eoff[k], eoff[k+1]) of src/dst with LOCAL vertex ids. voff/eoff hold
 * count+1 entries. Pass src = NULL to fill only the offsets.
 */
void gen_er_batch(int64_t count, const int64_t* vsizes, int64_t deg_num, int64_t deg_den,
                  uint64_t seed, int64_t* voff, int64_t* eoff, int32_t* src, int32_t* dst) {
    voff[0] = 0; eoff[0] = 0;
    for (int64_t k = 0; k < count; ++k) {
        voff[k + 1] = voff[k] + vsizes[k];
        eoff[k + 1] = eoff[k] + vsizes[k] * deg_num / deg_den;
    }
    if (!src) return;
    for (int64_t k = 0; k < count; ++k)
        gen_er(vsizes[k], eoff[k + 1] - eoff[k], derive(seed, 2000 + (uint64_t)k), src + eoff[k], dst + eoff[k]);
}

/*
 * Poisson job stream for a serving loop: inter-arrival gaps are exponential
 * with the given mean (seconds); kind[k] = 0 (list) with probability p_list,
 * else 1 (graph); sizes are log-uniform in [2^lo, 2^hi).
 */
void gen_jobs(int64_t count, double mean_gap, double p_list, double lo, double hi, uint64_t seed,
              double* arrival, int32_t* kind, int64_t* size) {
    uint64_t sa = derive(seed, 7), sk = derive(seed, 8), ss = derive(seed, 9);
    double t = 0.0;
    for (int64_t k = 0; k < count; ++k) {
        double u = to_unit(sm64_at(sa, (uint64_t)k + 1));
        t += -mean_gap * log(1.0 - u);
        arrival[k] = t;
        kind[k] = to_unit(sm64_at(sk, (uint64_t)k + 1)) < p_list ? 0 : 1;
        double w = to_unit(sm64_at(ss, (uint64_t)k + 1));
        int64_t v = (int64_t)floor(pow(2.0, lo + (hi - lo) * w));
        size[k] = v < 1 ? 1 : v;
    }
}

/*
 * The graph families of the paper's component experiments (Sec. 4: list
 * graphs, trees of degree k, random graphs of edge density d), as read here.
 * Vertex ids are a random permutation of [0, count*size), so each structure
 * sits at random places of the id space.
 *
 * List graph: count paths of `size` vertices; edge (perm[c*size+i],
 * perm[c*size+i+1]) joins consecutive vertices of path c.
 * m = count * (size - 1).
 */
int gen_list_graph(int64_t count, int64_t size, uint64_t seed, int32_t* src, int32_t* dst) {
    const int64_t n = count * size;
    int32_t* perm = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!perm) return 2;
    gen_permutation(n, derive(seed, 11), perm);
    int64_t e = 0;
    for (int64_t c = 0; c < count; ++c)
        for (int64_t i = 0; i + 1 < size; ++i, ++e) {
            src[e] = perm[c * size + i];
            dst[e] = perm[c * size + i + 1];
        }
    free(perm);
    return 0;
}

/*
 * Tree graph: count random trees of `size` vertices and degree k (at most k
 * children per vertex). Each tree grows one vertex at a time: vertex t takes
 * a child slot drawn uniformly from the open slots of vertices 0..t-1 (every
 * vertex brings k slots), the random recursive tree with bounded degree.
 * Edge (child, parent); m = count * (size - 1).
 */
int gen_tree_graph(int64_t count, int64_t size, int64_t k, uint64_t seed, int32_t* src, int32_t* dst) {
    if (k < 1) return 1;
    const int64_t n = count * size;
    int32_t* perm = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* slots = (int32_t*)malloc((size_t)(size * k + 1) * sizeof(int32_t));
    if (!perm || !slots) { free(perm); free(slots); return 2; }
    gen_permutation(n, derive(seed, 12), perm);
    sm64 g = { derive(seed, 13) };
    int64_t e = 0;
    for (int64_t c = 0; c < count; ++c) {
        const int32_t* id = perm + c * size;
        int64_t open = 0;
        for (int64_t j = 0; j < k; ++j) slots[open++] = 0;      /* the root's slots */
        for (int64_t t = 1; t < size; ++t, ++e) {
            const int64_t r = (int64_t)sm64_bounded(&g, (uint64_t)open);
            const int32_t parent = slots[r];
            slots[r] = slots[--open];
            src[e] = id[t];
            dst[e] = id[parent];
            for (int64_t j = 0; j < k; ++j) slots[open++] = (int32_t)t;
        }
    }
    free(perm);
    free(slots);
    return 0;
}

/* Raw access to the stream for tests of the generator itself. */
uint64_t gen_splitmix64_at(uint64_t seed, uint64_t k) { return sm64_at(seed, k); }
