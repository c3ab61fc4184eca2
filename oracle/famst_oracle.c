/*
 * FAMST CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct restatement of the FAMST method
 * (Almansoori & Telek, "FAMST: Fast Approximate Minimum Spanning Tree
 * Construction for Large-Scale and High-Dimensional Data"):
 *   Algorithm 1 (the driver), Algorithm 2 (undirected graph + DFS components),
 *   Algorithm 3 (lambda^2 random samples per component pair, keep lambda
 *   shortest), Algorithm 4 (neighbourhood refinement of inter-component
 *   edges), Kruskal's algorithm (Sec. 2.1 and the end of Sec. 3), the
 *   relative error of Eq. 1 against an exact MST, computed here by O(n^2)
 *   Prim instead of the dual-tree Boruvka EMST the paper uses.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this code. It shares nothing with the CUDA library; neither includes
 * nor links the other.
 *
 * Precision. The paper does not state one. Every decision (kNN order,
 * sample order, refinement comparisons, Kruskal order) is taken on the
 * canonical FP32 Euclidean distance: 32 partial sums, partial l taking the
 * coordinates t = l, l+32, l+64, ... < d in increasing order,
 *     p_l = 0;  p_l = fmaf(delta_t, delta_t, p_l),  delta_t = x[t] - y[t]
 * then combined pairwise by the butterfly o = 16, 8, 4, 2, 1:
 *     p_l <- p_l + p_(l xor o)   (every l at once; lane 0's value is kept)
 *     w = sqrtf(p_0)
 * (fmaf, + and sqrtf are correctly rounded; build with -ffp-contract=off).
 * This is the order a 32-lane warp evaluates naturally; it is symmetric in
 * x and y bit for bit.
 * Sums of weights are taken in double. dist64() is the same distance in
 * double precision, used for the FP64 tree weight and the gradient.
 *
 * Total order of edges: (w, min(u,v), max(u,v)) ascending; of neighbours of
 * a row: (w, id) ascending; of samples of a component pair: (w, sample index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- distance */

float or_dist32(const float *a, const float *b, int d)
{
    float p[32], q[32];
    for (int l = 0; l < 32; ++l) p[l] = 0.0f;
    for (int t = 0; t < d; ++t) {        /* partial t mod 32, t increasing */
        float delta = a[t] - b[t];
        p[t & 31] = fmaf(delta, delta, p[t & 31]);
    }
    for (int o = 16; o >= 1; o >>= 1) {  /* butterfly, all partials at once */
        for (int l = 0; l < 32; ++l) q[l] = p[l] + p[l ^ o];
        for (int l = 0; l < 32; ++l) p[l] = q[l];
    }
    return sqrtf(p[0]);
}

double or_dist64(const float *a, const float *b, int d)
{
    double p = 0.0;
    for (int t = 0; t < d; ++t) {
        double delta = (double)a[t] - (double)b[t];
        p += delta * delta;
    }
    return sqrt(p);
}

/* (w, j) < (w2, j2) in lexicographic order */
static int nb_less(float w, int j, float w2, int j2)
{
    return (w < w2) || (w == w2 && j < j2);
}

/* ---------------------------------------------------- Phase 1: exact kNN
 * GetANNs (Algorithm 1, first step) realised as brute force: for every query
 * row i in [r0, r1) the k smallest (w(i,j), j) over all j != i, ascending.
 * Output rows are relative to r0: nbr[(i - r0) * k + r]. */
void or_knn(const float *X, int64_t n, int d, int k, int64_t r0, int64_t r1,
            int32_t *nbr, float *dist, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t i = r0; i < r1; ++i) {
        int32_t *ni = nbr + (i - r0) * k;
        float *di = dist + (i - r0) * k;
        int have = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            float w = or_dist32(X + i * d, X + j * d, d);
            if (have == k && !nb_less(w, (int)j, di[k - 1], ni[k - 1]))
                continue;
            /* insertion into the sorted list */
            int pos = have < k ? have : k - 1;
            while (pos > 0 && nb_less(w, (int)j, di[pos - 1], ni[pos - 1])) {
                di[pos] = di[pos - 1];
                ni[pos] = ni[pos - 1];
                --pos;
            }
            di[pos] = w;
            ni[pos] = (int32_t)j;
            if (have < k) ++have;
        }
    }
}

/* ---------------------------------------- Phase 2a: graph and components */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Algorithm 2, first loop: for each i and each j in N[i] add (i,j) and
 * (j,i) to G. Adjacency lists are deduplicated and sorted by id.
 * row_ptr has n+1 entries; col must hold 2*n*k entries. Returns nnz. */
int64_t or_build_graph(const int32_t *nbr, int64_t n, int k, int64_t *row_ptr,
                       int32_t *col)
{
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < k; ++r) {
            int32_t j = nbr[i * k + r];
            deg[i]++;
            deg[j]++;
        }
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i];
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < k; ++r) {
            int32_t j = nbr[i * k + r];
            col[row_ptr[i] + fill[i]++] = j;
            col[row_ptr[j] + fill[j]++] = (int32_t)i;
        }
    /* sort and deduplicate each list, compacting in place */
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = row_ptr[i], b = row_ptr[i + 1];
        qsort(col + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        row_ptr[i] = out;
        for (int64_t e = a; e < b; ++e)
            if (e == a || col[e] != col[e - 1]) col[out++] = col[e];
    }
    row_ptr[n] = out;
    free(deg);
    free(fill);
    return out;
}

/* Algorithm 2, DFS part: visit vertices i = 0, 1, ... ; an unvisited i
 * starts a new component c' explored with an explicit stack. comp[v]
 * receives the component's index in discovery order. members / comp_off
 * list each component's vertices sorted by id (comp_off has t+1 entries,
 * the caller sizes it n+1). Returns t. */
int64_t or_components(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      int32_t *comp, int32_t *members, int64_t *comp_off)
{
    unsigned char *visited = (unsigned char *)calloc((size_t)n, 1);
    int64_t nnz = row_ptr[n];
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz + n + 1));
    int64_t t = 0, filled = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (visited[i]) continue;
        comp_off[t] = filled;
        int64_t sp = 0;
        stack[sp++] = (int32_t)i;
        while (sp > 0) {
            int32_t u = stack[--sp];
            if (visited[u]) continue;
            visited[u] = 1;
            comp[u] = (int32_t)t;
            members[filled++] = u;
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                if (!visited[col[e]]) stack[sp++] = col[e];
        }
        qsort(members + comp_off[t], (size_t)(filled - comp_off[t]),
              sizeof(int32_t), cmp_i32);
        ++t;
    }
    comp_off[t] = filled;
    free(visited);
    free(stack);
    return t;
}

/* ------------------------------------------------------- Philox4x32-10
 * Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
 *   (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
 * with the key bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform index in [0, size) from a 32-bit draw (multiply-shift) */
static int64_t pick(uint32_t r, int64_t size)
{
    return (int64_t)(((uint64_t)r * (uint64_t)size) >> 32);
}

/* ------------------------------------ Phase 1 alternative: NN-Descent
 * GetANNs by NN-Descent (Dong, Charikar and Li, WWW 2011), the algorithm of
 * the library the paper uses for its Phase 1 (Sec. 2 and Sec. 3). Every step
 * is defined on sets, so the result does not depend on the order in which
 * the comparisons are made; draws come from Philox4x32-10 with the key
 * (seed_lo, seed_hi):
 *
 * Lists. B[v] holds k distinct ids u != v with (w(v,u), u) ascending and a
 *   flag "new" per entry.
 * Start. Without a given graph, B[v] takes the first k distinct ids among
 *   the draws r = 0 .. 8k-1, u = pick(r0, n-1) (u += 1 when u >= v) with
 *   (r0, ., ., .) = Philox(counter = (v, r, 0, 1)); if fewer than k are
 *   distinct, the smallest unused ids fill the list. Every entry is new.
 * One iteration (it = 0, 1, ...), on the lists as the iteration finds them:
 *   1. For every v and each class (new, old): the candidates are the ids
 *      u of B[v] of that class and the ids u whose list B[u] holds v with
 *      that class; each candidate has the priority
 *      pr(v,u) = r0 of Philox(counter = (v, u, it, 2)), and the S candidates
 *      smallest in (pr, u) form new[v] (resp. old[v]): the sample of rate
 *      S / k of the paper, taken jointly over both directions.
 *   2. Every entry u of B[v] that is new and in new[v] becomes old.
 *   3. Local join: for every v, each pair of distinct ids {a, b} with a, b
 *      in new[v], or a in new[v] and b in old[v], proposes b to B[a] and a
 *      to B[b] with w(a, b).
 *   4. B[a] becomes the k smallest distinct (w, id) of B[a] and every
 *      proposal to a; an entry that came from a proposal is new.
 *   c = the number of entries in all lists that were not there before.
 * The iterations stop after the first one with c = 0 or c < delta n k, or
 * after max_iters. Returns the number of iterations run; updates[it] = c and
 * pairs[it] = the pairs {a, b} (a != b) its joins evaluated, counted once
 * per v and per set they came from: C(|new[v]|, 2) + |new[v] x old[v]|
 * less the pairs with a = b. */
typedef struct { float w; int32_t id; uint8_t flag; } nnd_ent;
enum { NND_NEW = 1, NND_INSERTED = 2 };
typedef struct { uint32_t pr; int32_t u; } nnd_cand;

static uint32_t nnd_draw(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         const uint32_t key[2])
{
    uint32_t ctr[4] = {c0, c1, c2, c3}, r[4];
    or_philox4x32_10(ctr, key, r);
    return r[0];
}

static int cmp_nnd_cand(const void *a, const void *b)
{
    const nnd_cand *x = (const nnd_cand *)a, *y = (const nnd_cand *)b;
    if (x->pr != y->pr) return x->pr < y->pr ? -1 : 1;
    return (x->u > y->u) - (x->u < y->u);
}

/* insert (w, id) into the sorted list L of k entries if it is among the k
 * smallest and not already there */
static void nnd_insert(nnd_ent *L, int k, float w, int32_t id)
{
    if (!nb_less(w, id, L[k - 1].w, L[k - 1].id)) return;
    for (int r = 0; r < k; ++r)
        if (L[r].id == id) return;
    int pos = k - 1;
    while (pos > 0 && nb_less(w, id, L[pos - 1].w, L[pos - 1].id)) {
        L[pos] = L[pos - 1];
        --pos;
    }
    L[pos].w = w;
    L[pos].id = id;
    L[pos].flag = NND_NEW | NND_INSERTED;
}

int or_nndescent(const float *X, int64_t n, int d, int k, int S, int max_iters,
                 double delta, uint64_t seed, const int32_t *init,
                 int32_t *nbr, float *dist, int64_t *updates, int64_t *pairs)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    nnd_ent *B = (nnd_ent *)malloc(sizeof(nnd_ent) * (size_t)(n * k));
    /* start */
    for (int64_t v = 0; v < n; ++v) {
        nnd_ent *L = B + v * k;
        int have = 0;
        if (init) {
            for (int r = 0; r < k; ++r) L[r].id = init[v * k + r];
            have = k;
        }
        for (int r = 0; r < 8 * k && have < k; ++r) {
            int64_t u = pick(nnd_draw((uint32_t)v, (uint32_t)r, 0u, 1u, key), n - 1);
            if (u >= v) ++u;
            int dup = 0;
            for (int q = 0; q < have; ++q) dup |= L[q].id == (int32_t)u;
            if (!dup) L[have++].id = (int32_t)u;
        }
        for (int64_t u = 0; u < n && have < k; ++u) {
            int dup = u == v;
            for (int q = 0; q < have; ++q) dup |= L[q].id == (int32_t)u;
            if (!dup) L[have++].id = (int32_t)u;
        }
        for (int r = 0; r < k; ++r) {
            L[r].w = or_dist32(X + v * d, X + (int64_t)L[r].id * d, d);
            L[r].flag = NND_NEW;
        }
        for (int r = 1; r < k; ++r) {   /* insertion sort by (w, id) */
            nnd_ent e = L[r];
            int q = r;
            while (q > 0 && nb_less(e.w, e.id, L[q - 1].w, L[q - 1].id)) {
                L[q] = L[q - 1];
                --q;
            }
            L[q] = e;
        }
    }
    int32_t *samp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n * S));
    int32_t *scnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
    int64_t *roff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * (n + 1)));
    int32_t *rsrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * k));
    nnd_cand *cbuf = (nnd_cand *)malloc(sizeof(nnd_cand) * (size_t)(n * k + k));
    float *wbuf = (float *)malloc(sizeof(float) * (size_t)(1024 * ((int64_t)S * (3 * S - 1) / 2)));
    int it = 0;
    while (it < max_iters) {
        /* step 1: reverse entries of each class, by counting */
        for (int cls = 0; cls < 2; ++cls) {
            int64_t *off = roff + cls * (n + 1);
            for (int64_t v = 0; v <= n; ++v) off[v] = 0;
            for (int64_t e = 0; e < n * k; ++e)
                if (((B[e].flag & NND_NEW) != 0) == (cls == 0)) off[B[e].id + 1] += 1;
            for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
        }
        for (int cls = 0; cls < 2; ++cls) {
            const int64_t *off = roff + cls * (n + 1);
            int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
            for (int64_t e = 0; e < n * k; ++e) {
                if (((B[e].flag & NND_NEW) != 0) != (cls == 0)) continue;
                int32_t v = B[e].id;
                rsrc[off[v] + fill[v]++] = (int32_t)(e / k);
            }
            free(fill);
            for (int64_t v = 0; v < n; ++v) {
                int m = 0;
                for (int r = 0; r < k; ++r) {
                    const nnd_ent *x = B + v * k + r;
                    if (((x->flag & NND_NEW) != 0) == (cls == 0)) cbuf[m++].u = x->id;
                }
                for (int64_t q = off[v]; q < off[v + 1]; ++q) cbuf[m++].u = rsrc[q];
                for (int q = 0; q < m; ++q)
                    cbuf[q].pr = nnd_draw((uint32_t)v, (uint32_t)cbuf[q].u, (uint32_t)it, 2u, key);
                qsort(cbuf, (size_t)m, sizeof(nnd_cand), cmp_nnd_cand);
                int c = 0;
                for (int q = 0; q < m && c < S; ++q) {
                    if (q > 0 && cbuf[q].u == cbuf[q - 1].u) continue;   /* both directions */
                    samp[(cls * n + v) * S + c++] = cbuf[q].u;
                }
                scnt[cls * n + v] = c;
            }
        }
        /* step 2 */
        for (int64_t v = 0; v < n; ++v) {
            const int32_t *nv = samp + v * S;
            for (int r = 0; r < k; ++r) {
                nnd_ent *x = B + v * k + r;
                if (!(x->flag & NND_NEW)) continue;
                for (int q = 0; q < scnt[v]; ++q)
                    if (nv[q] == x->id) x->flag = 0;
            }
        }
        /* steps 3 and 4: the lists are updated as proposals arrive, which
         * gives the k smallest of the union whatever the order; the
         * distances of a block of joins are computed first, spread over
         * threads (they do not depend on the lists) */
        const int64_t VB = 1024, PP = (int64_t)S * (3 * S - 1) / 2;
        int64_t joined = 0;
        for (int64_t v0 = 0; v0 < n; v0 += VB) {
            const int64_t v1 = v0 + VB < n ? v0 + VB : n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
            for (int64_t v = v0; v < v1; ++v) {
                const int32_t *nv = samp + v * S, *ov = samp + (n + v) * S;
                const int nn = scnt[v], no = scnt[n + v];
                float *wv = wbuf + (v - v0) * PP;
                int64_t q = 0;
                for (int i = 0; i < nn; ++i) {
                    const float *xa = X + (int64_t)nv[i] * d;
                    for (int j = i + 1; j < nn; ++j)
                        wv[q++] = or_dist32(xa, X + (int64_t)nv[j] * d, d);
                    for (int j = 0; j < no; ++j)
                        wv[q++] = or_dist32(xa, X + (int64_t)ov[j] * d, d);
                }
            }
            for (int64_t v = v0; v < v1; ++v) {
                const int32_t *nv = samp + v * S, *ov = samp + (n + v) * S;
                const int nn = scnt[v], no = scnt[n + v];
                const float *wv = wbuf + (v - v0) * PP;
                int64_t q = 0;
                for (int i = 0; i < nn; ++i) {
                    const int32_t a = nv[i];
                    for (int j = i + 1; j < nn; ++j, ++q) {
                        ++joined;
                        nnd_insert(B + (int64_t)a * k, k, wv[q], nv[j]);
                        nnd_insert(B + (int64_t)nv[j] * k, k, wv[q], a);
                    }
                    for (int j = 0; j < no; ++j, ++q) {
                        if (ov[j] == a) continue;   /* a in both samples */
                        ++joined;
                        nnd_insert(B + (int64_t)a * k, k, wv[q], ov[j]);
                        nnd_insert(B + (int64_t)ov[j] * k, k, wv[q], a);
                    }
                }
            }
        }
        int64_t c = 0;
        for (int64_t e = 0; e < n * k; ++e) {
            c += (B[e].flag & NND_INSERTED) != 0;
            B[e].flag &= (uint8_t)~NND_INSERTED;
        }
        if (updates) updates[it] = c;
        if (pairs) pairs[it] = joined;
        ++it;
        if (c == 0 || (double)c < delta * (double)n * (double)k) break;
    }
    for (int64_t e = 0; e < n * k; ++e) {
        nbr[e] = B[e].id;
        dist[e] = B[e].w;
    }
    free(B);
    free(samp);
    free(scnt);
    free(roff);
    free(rsrc);
    free(cbuf);
    free(wbuf);
    return it;
}

typedef struct { float w; int32_t s; int32_t u; int32_t v; } sample_t;

static int cmp_sample(const void *a, const void *b)
{
    const sample_t *x = (const sample_t *)a, *y = (const sample_t *)b;
    if (x->w < y->w) return -1;
    if (x->w > y->w) return 1;
    return (x->s > y->s) - (x->s < y->s);
}

/* ------------------------------------------------ Phase 2b: Algorithm 3
 * For every component pair i < j (i outer, j inner, both in discovery
 * order) draw lambda^2 samples s = 0 .. lambda^2-1:
 *   (r0, r1, ., .) = Philox4x32-10(counter = (s, p_lo, p_hi, 0),
 *                                  key = (seed_lo, seed_hi)),  p = i*t + j
 *   u = C_i[pick(r0, |C_i|)],  v = C_j[pick(r1, |C_j|)],  d = w(u, v)
 * sort the samples by (d, s) and append the first lambda to E, with
 * (i, j) to E_C. Members C_i are sorted by id. Returns |E|. */
int64_t or_random_edges(const float *X, int d, const int32_t *members,
                        const int64_t *comp_off, int64_t t, int lambda,
                        uint64_t seed, int32_t *eu, int32_t *ev, float *ew,
                        int32_t *eci, int32_t *ecj)
{
    int L2 = lambda * lambda;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    /* pairs are drawn and selected independently of each other (Alg. 3), so
     * the outer loop is spread over threads; pair (i, j) writes its lambda
     * edges at its rank in the (i outer, j inner) order */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < t; ++i) {
        sample_t *cand = (sample_t *)malloc(sizeof(sample_t) * (size_t)L2);
        int64_t m = (i * t - i * (i + 1) / 2) * lambda;
        for (int64_t j = i + 1; j < t; ++j) {
            uint64_t p = (uint64_t)i * (uint64_t)t + (uint64_t)j;
            int64_t si = comp_off[i + 1] - comp_off[i];
            int64_t sj = comp_off[j + 1] - comp_off[j];
            for (int s = 0; s < L2; ++s) {
                uint32_t ctr[4] = {(uint32_t)s, (uint32_t)p, (uint32_t)(p >> 32), 0u};
                uint32_t r[4];
                or_philox4x32_10(ctr, key, r);
                int32_t u = members[comp_off[i] + pick(r[0], si)];
                int32_t v = members[comp_off[j] + pick(r[1], sj)];
                cand[s].w = or_dist32(X + (int64_t)u * d, X + (int64_t)v * d, d);
                cand[s].s = s;
                cand[s].u = u;
                cand[s].v = v;
            }
            qsort(cand, (size_t)L2, sizeof(sample_t), cmp_sample);
            for (int r = 0; r < lambda; ++r) {
                eu[m] = cand[r].u;
                ev[m] = cand[r].v;
                ew[m] = cand[r].w;
                eci[m] = (int32_t)i;
                ecj[m] = (int32_t)j;
                ++m;
            }
        }
        free(cand);
    }
    return lambda * t * (t - 1) / 2;
}

/* ------------------------- Phase 2b variant: the lambda nearest pairs
 * The variant of Algorithm 3 that joins components by their nearest
 * pairs instead of random samples ("the lambda nearest cross-component
 * edges"): for every component pair i < j (i outer, j inner), all
 * |C_i| |C_j| pairs (u in C_i, v in C_j) are compared by the canonical
 * distance and the lambda smallest under the edge order (w, min(u,v),
 * max(u,v)) are kept, ascending. Edge e = (pair rank) * lambda + r holds
 * (u, v, w, i, j). A component pair with fewer than lambda cross pairs
 * repeats its farthest pair in the remaining slots (duplicate edges change
 * neither the refinement nor Kruskal). Returns |E| = lambda t (t - 1) / 2. */
typedef struct { float w; int32_t a; int32_t b; int32_t u; int32_t v; } pairkey_t;

static int pair_less(const pairkey_t *x, const pairkey_t *y)
{
    if (x->w != y->w) return x->w < y->w;
    if (x->a != y->a) return x->a < y->a;
    return x->b < y->b;
}

int64_t or_nearest_edges(const float *X, int d, const int32_t *members,
                         const int64_t *comp_off, int64_t t, int lambda,
                         int32_t *eu, int32_t *ev, float *ew, int32_t *eci,
                         int32_t *ecj)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < t; ++i) {
        pairkey_t *best = (pairkey_t *)malloc(sizeof(pairkey_t) * (size_t)lambda);
        for (int64_t j = i + 1; j < t; ++j) {
            int have = 0;
            for (int64_t a = comp_off[i]; a < comp_off[i + 1]; ++a) {
                for (int64_t b = comp_off[j]; b < comp_off[j + 1]; ++b) {
                    pairkey_t c;
                    c.u = members[a];
                    c.v = members[b];
                    c.w = or_dist32(X + (int64_t)c.u * d, X + (int64_t)c.v * d, d);
                    c.a = c.u < c.v ? c.u : c.v;
                    c.b = c.u < c.v ? c.v : c.u;
                    if (have == lambda && !pair_less(&c, &best[lambda - 1])) continue;
                    int pos = have < lambda ? have : lambda - 1;   /* sorted insertion */
                    while (pos > 0 && pair_less(&c, &best[pos - 1])) {
                        best[pos] = best[pos - 1];
                        --pos;
                    }
                    best[pos] = c;
                    if (have < lambda) ++have;
                }
            }
            int64_t base = (i * t - i * (i + 1) / 2 + (j - i - 1)) * lambda;
            for (int r = 0; r < lambda; ++r) {
                const pairkey_t *c = &best[r < have ? r : have - 1];
                eu[base + r] = c->u;
                ev[base + r] = c->v;
                ew[base + r] = c->w;
                eci[base + r] = (int32_t)i;
                ecj[base + r] = (int32_t)j;
            }
        }
        free(best);
    }
    return lambda * t * (t - 1) / 2;
}

/* --------------------------------------------------- Phase 3: Algorithm 4
 * One refinement sweep over E, in place (edges do not depend on each
 * other). For edge (u, v, d) of pair (C_i, C_j):
 *   u*, v*, d* = u, v, d
 *   for u' in G[u] with comp[u'] == i, ascending:   if u' != v and
 *       w(u', v) < d*:  u* = u', d* = w(u', v)
 *   for v' in G[v] with comp[v'] == j, ascending:   if v' != u and
 *       w(u*, v') < d*: v* = v', d* = w(u*, v')
 *   the edge becomes (u*, v*, d*); it counts in Delta if (u*,v*) != (u,v).
 * changed[e] (optional) receives 1 for edges in Delta. Returns |Delta|. */
int64_t or_refine_sweep(const float *X, int d, const int64_t *row_ptr,
                        const int32_t *col, const int32_t *comp, int64_t m,
                        int32_t *eu, int32_t *ev, float *ew,
                        const int32_t *eci, const int32_t *ecj,
                        unsigned char *changed)
{
    int64_t delta = 0;
    /* an edge's update reads only its own (u, v, d) and the fixed X, G and
     * labels (Alg. 4), so edges are spread over threads */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) reduction(+:delta)
#endif
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = eu[e], v = ev[e];
        int32_t us = u, vs = v;
        float ds = ew[e];
        for (int64_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q) {
            int32_t up = col[q];
            if (comp[up] != eci[e]) continue;
            if (up == v) continue;
            float dp = or_dist32(X + (int64_t)up * d, X + (int64_t)v * d, d);
            if (dp < ds) { us = up; ds = dp; }
        }
        for (int64_t q = row_ptr[v]; q < row_ptr[v + 1]; ++q) {
            int32_t vp = col[q];
            if (comp[vp] != ecj[e]) continue;
            if (vp == u) continue;
            float dp = or_dist32(X + (int64_t)us * d, X + (int64_t)vp * d, d);
            if (dp < ds) { vs = vp; ds = dp; }
        }
        int ch = (us != u) || (vs != v);
        if (changed) changed[e] = (unsigned char)ch;
        delta += ch;
        eu[e] = us;
        ev[e] = vs;
        ew[e] = ds;
    }
    return delta;
}

/* ------------------------------------------------------------ Kruskal */

typedef struct { float w; int32_t a; int32_t b; } edge_t; /* a < b */

static int cmp_edge(const void *x, const void *y)
{
    const edge_t *p = (const edge_t *)x, *q = (const edge_t *)y;
    if (p->w < q->w) return -1;
    if (p->w > q->w) return 1;
    if (p->a != q->a) return (p->a > q->a) - (p->a < q->a);
    return (p->b > q->b) - (p->b < q->b);
}

static int32_t uf_find(int32_t *par, int32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

/* Kruskal's algorithm (Sec. 2.1) on the union of the kNN edges
 * {i, nbr[i][r]} weighted by dist[i][r] and the m edges of E: sort all
 * edges by (w, min id, max id), scan them, keep an edge when its end points
 * are in different sets and merge the sets. Tree edges are written in the
 * order Kruskal accepts them, as (min id, max id, w); W is their sum in
 * double, in that order. Returns the number of tree edges. */
int64_t or_kruskal(int64_t n, const int32_t *nbr, const float *dist, int k,
                   int64_t m, const int32_t *eu, const int32_t *ev,
                   const float *ew, int32_t *tu, int32_t *tv, float *tw,
                   double *W)
{
    int64_t total = n * (int64_t)k + m;
    edge_t *all = (edge_t *)malloc(sizeof(edge_t) * (size_t)(total > 0 ? total : 1));
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < k; ++r) {
            int32_t j = nbr[i * k + r];
            all[c].w = dist[i * k + r];
            all[c].a = (int32_t)(i < j ? i : j);
            all[c].b = (int32_t)(i < j ? j : i);
            ++c;
        }
    for (int64_t e = 0; e < m; ++e) {
        all[c].w = ew[e];
        all[c].a = eu[e] < ev[e] ? eu[e] : ev[e];
        all[c].b = eu[e] < ev[e] ? ev[e] : eu[e];
        ++c;
    }
    qsort(all, (size_t)total, sizeof(edge_t), cmp_edge);
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) par[i] = (int32_t)i;
    int64_t got = 0;
    double sum = 0.0;
    for (int64_t e = 0; e < total && got < n - 1; ++e) {
        int32_t ra = uf_find(par, all[e].a), rb = uf_find(par, all[e].b);
        if (ra == rb) continue;
        par[ra] = rb;
        tu[got] = all[e].a;
        tv[got] = all[e].b;
        tw[got] = all[e].w;
        sum += (double)all[e].w;
        ++got;
    }
    *W = sum;
    free(all);
    free(par);
    return got;
}

/* ------------------------------------------------- exact MST by Prim
 * O(n^2) Prim on the complete graph with canonical FP32 weights and the
 * edge order (w, min id, max id); the tree it returns is the unique MST
 * under that order. It plays the role of the exact EMST in Eq. 1. Tree
 * edges come out in the order Prim adds them, as (min id, max id, w). */
static int key_less(float w, int32_t a, int32_t b, float w2, int32_t a2, int32_t b2)
{
    if (w != w2) return w < w2;
    if (a != a2) return a < a2;
    return b < b2;
}

void or_prim(const float *X, int64_t n, int d, int32_t *tu, int32_t *tv,
             float *tw, double *W, int threads)
{
    if (n <= 1) { *W = 0.0; return; }
    unsigned char *in_tree = (unsigned char *)calloc((size_t)n, 1);
    float *bw = (float *)malloc(sizeof(float) * (size_t)n);
    int32_t *ba = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *bb = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) { bw[v] = INFINITY; ba[v] = bb[v] = INT32_MAX; }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    int64_t last = 0;
    in_tree[0] = 1;
    double sum = 0.0;
    for (int64_t step = 0; step < n - 1; ++step) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t v = 0; v < n; ++v) {
            if (in_tree[v]) continue;
            float w = or_dist32(X + last * d, X + v * d, d);
            int32_t a = (int32_t)(last < v ? last : v), b = (int32_t)(last < v ? v : last);
            if (key_less(w, a, b, bw[v], ba[v], bb[v])) { bw[v] = w; ba[v] = a; bb[v] = b; }
        }
        int64_t best = -1;
        for (int64_t v = 0; v < n; ++v) {
            if (in_tree[v]) continue;
            if (best < 0 || key_less(bw[v], ba[v], bb[v], bw[best], ba[best], bb[best]))
                best = v;
        }
        in_tree[best] = 1;
        tu[step] = ba[best];
        tv[step] = bb[best];
        tw[step] = bw[best];
        sum += (double)bw[best];
        last = best;
    }
    *W = sum;
    free(in_tree); free(bw); free(ba); free(bb);
}

/* ------------------------------------------- weights and the gradient */

/* FP64 weight of a tree: sum of dist64 over its edges, in edge order. */
double or_tree_weight64(const float *X, int d, const int32_t *tu,
                        const int32_t *tv, int64_t m)
{
    double s = 0.0;
    for (int64_t e = 0; e < m; ++e)
        s += or_dist64(X + (int64_t)tu[e] * d, X + (int64_t)tv[e] * d, d);
    return s;
}

/* Gradient of W = sum over tree edges of ||x_u - x_v|| with the tree held
 * fixed: dW/dx_u += (x_u - x_v)/||x_u - x_v||, dW/dx_v -= the same, in
 * double; an edge of length zero contributes zero. g is n x d, zeroed
 * here. */
void or_mst_grad(const float *X, int64_t n, int d, const int32_t *tu,
                 const int32_t *tv, int64_t m, double *g)
{
    memset(g, 0, sizeof(double) * (size_t)(n * d));
    for (int64_t e = 0; e < m; ++e) {
        const float *xu = X + (int64_t)tu[e] * d, *xv = X + (int64_t)tv[e] * d;
        double w = or_dist64(xu, xv, d);
        if (w == 0.0) continue;
        for (int t = 0; t < d; ++t) {
            double q = ((double)xu[t] - (double)xv[t]) / w;
            g[(int64_t)tu[e] * d + t] += q;
            g[(int64_t)tv[e] * d + t] -= q;
        }
    }
}
