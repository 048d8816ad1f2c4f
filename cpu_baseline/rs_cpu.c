/*
 * Multi-threaded CPU list ranking by random splitters (the paper's CPU
 * comparison point, Sec. 3.2: the same sparse ruling set, run by threads on
 * the host cores). A timed baseline for the benchmark; it shares no code with
 * the CUDA library or the oracle.
 *
 *   1. splitters: the head plus one element at a random offset in every block
 *      of D consecutive ids (offsets from SplitMix64, Steele et al. 2014);
 *   2. every thread walks the sublists of its share of the splitters, giving
 *      each visited element its owner and its position in the sublist, and
 *      records each sublist's length and the splitter that ends it;
 *   3. one thread ranks the splitter list by walking it from the head;
 *   4. every thread expands its share of the elements:
 *      rank = (elements from the owner to the tail) - 1 - position.
 *
 * Returns 0 on success, 1 on a bad argument or allocation failure, 4 when the
 * input is not a single list.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const int32_t* succ;
    int64_t n, D, nb;
    int32_t head;
    int32_t* spl_of;     /* splitter index of element i, or -1 */
    int32_t* spl_elem;   /* element of splitter j */
    int32_t* owner;      /* owner splitter of element i */
    int32_t* pos;        /* position of element i in its sublist (splitter: 0) */
    int32_t* nextspl;    /* splitter that ends sublist j, or -1 at the tail */
    int32_t* len;        /* elements of sublist j, its splitter included */
    int32_t* srank;      /* elements from splitter j to the tail */
    int32_t* rank;
    uint64_t seed;
    int threads;
    volatile int bad;
} job_t;

typedef struct { job_t* job; int t; int phase; } arg_t;

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void range_of(int64_t total, int threads, int t, int64_t* b, int64_t* e) {
    *b = total * t / threads;
    *e = total * (t + 1) / threads;
}

static void* run_phase(void* p) {
    arg_t* a = (arg_t*)p;
    job_t* J = a->job;
    int64_t b, e;
    if (a->phase == 0) {                       /* choose splitters: one per block of D ids */
        range_of(J->nb, J->threads, a->t, &b, &e);
        const int64_t hb = J->head / J->D;
        for (int64_t blk = b; blk < e; ++blk) {
            const int64_t lo = blk * J->D;
            const int64_t sz = (lo + J->D <= J->n) ? J->D : J->n - lo;
            int64_t el = (blk == hb) ? J->head
                         : lo + (int64_t)((mix64(J->seed + 0x9e3779b97f4a7c15ULL * (uint64_t)(blk + 1)) >> 11) % (uint64_t)sz);
            /* splitter index: blocks numbered from the head's block, so the head is splitter 0 */
            const int64_t j = blk >= hb ? blk - hb : blk - hb + J->nb;
            J->spl_of[el] = (int32_t)j;
            J->spl_elem[j] = (int32_t)el;
        }
    } else if (a->phase == 1) {                /* walk the sublists of this thread's splitters */
        range_of(J->nb, J->threads, a->t, &b, &e);
        for (int64_t j = b; j < e && !J->bad; ++j) {
            int64_t cur = J->spl_elem[j];
            int32_t k = 0;
            for (;;) {
                J->owner[cur] = (int32_t)j;
                J->pos[cur] = k++;
                const int64_t nx = J->succ[cur];
                if (nx == -1 || nx == cur) { J->nextspl[j] = -1; break; }
                if (nx < 0 || nx >= J->n || k > J->n) { J->bad = 1; break; }
                if (J->spl_of[nx] >= 0) { J->nextspl[j] = J->spl_of[nx]; break; }
                cur = nx;
            }
            J->len[j] = k;
        }
    } else {                                   /* expand this thread's share of the elements */
        range_of(J->n, J->threads, a->t, &b, &e);
        for (int64_t i = b; i < e; ++i) J->rank[i] = J->srank[J->owner[i]] - 1 - J->pos[i];
    }
    return NULL;
}

static int run_threads(job_t* J, int phase) {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)J->threads);
    arg_t* args = (arg_t*)malloc(sizeof(arg_t) * (size_t)J->threads);
    if (!th || !args) { free(th); free(args); return 1; }
    for (int t = 0; t < J->threads; ++t) {
        args[t].job = J; args[t].t = t; args[t].phase = phase;
        if (t == 0) continue;
        if (pthread_create(&th[t], NULL, run_phase, &args[t])) { J->bad = 2; args[t].phase = -1; }
    }
    run_phase(&args[0]);
    for (int t = 1; t < J->threads; ++t)
        if (args[t].phase >= 0) pthread_join(th[t], NULL);
    free(th);
    free(args);
    return J->bad == 2;
}

int cpu_lr_rank(const int32_t* succ, int64_t n, int32_t head, int32_t* rank, int threads, int64_t D,
                uint64_t seed) {
    if (n <= 0) return n == 0 ? 0 : 1;
    if (head < 0 || head >= n || threads < 1 || D < 1) return 1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.succ = succ; J.n = n; J.head = head; J.D = D; J.nb = (n + D - 1) / D;
    J.rank = rank; J.seed = seed; J.threads = threads;
    J.spl_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    J.owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    J.pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    J.spl_elem = (int32_t*)malloc(sizeof(int32_t) * (size_t)J.nb);
    J.nextspl = (int32_t*)malloc(sizeof(int32_t) * (size_t)J.nb);
    J.len = (int32_t*)malloc(sizeof(int32_t) * (size_t)J.nb);
    J.srank = (int32_t*)malloc(sizeof(int32_t) * (size_t)J.nb);
    int rc = 0;
    if (!J.spl_of || !J.owner || !J.pos || !J.spl_elem || !J.nextspl || !J.len || !J.srank) { rc = 1; goto done; }
    memset(J.spl_of, 0xff, sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) J.owner[i] = -1;
    if (run_threads(&J, 0) || run_threads(&J, 1)) { rc = 1; goto done; }
    if (J.bad) { rc = 4; goto done; }
    /* rank the splitter list: walk it from splitter 0, then suffix sums backwards */
    {
        int32_t* order = J.srank;              /* reused: splitters in list order */
        int64_t r = 0;
        int64_t total = 0;
        int64_t j = 0;
        for (; j >= 0 && r < J.nb; j = J.nextspl[j]) {
            order[r++] = (int32_t)j;
            total += J.len[j];
        }
        /* one list: every splitter once, ending at the tail (a cycle comes back instead) */
        if (j >= 0 || r != J.nb || total != n) { rc = 4; goto done; }
        int32_t* tmp = J.spl_of;               /* reused: no longer needed */
        int32_t acc = 0;
        for (int64_t q = r - 1; q >= 0; --q) {
            acc += J.len[order[q]];
            tmp[order[q]] = acc;
        }
        memcpy(J.srank, tmp, sizeof(int32_t) * (size_t)J.nb);
    }
    for (int64_t i = 0; i < n; ++i)
        if (J.owner[i] < 0) { rc = 4; goto done; }
    if (run_threads(&J, 2)) rc = 1;
done:
    free(J.spl_of); free(J.owner); free(J.pos); free(J.spl_elem); free(J.nextspl); free(J.len); free(J.srank);
    return rc;
}
