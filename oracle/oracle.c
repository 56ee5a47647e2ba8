/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.  Plain, sequential, obviously
 * correct CPU reference for ConnectIt's connectivity path (Dhulipala, Hong,
 * Shun, "ConnectIt: A Framework for Static and Incremental Parallel Graph
 * Connectivity Algorithms").  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path
 * never calls it and shares no code with it.
 *
 * Graph layout (Section 2, "Graph Notation and Formats"): CSR with offsets
 * I[0..n] (I[n] = m; the text's "A[n] = m" is read as I[n] = m) and edges
 * A[0..m-1]; the neighbours of v are A[I[v]] .. A[I[v+1]-1].  The graph is
 * symmetric (every undirected edge is stored in both directions).
 *
 * Result (Section 2, "Graph Connectivity"): a connectivity labelling, here
 * fixed to its canonical form label[v] = min{ u : u connected to v }, so it
 * is unique and a GPU result can be compared bit for bit.
 *
 * What each function follows:
 *   oracle_cc_uf          plain definition, by sequential union-find (O1)
 *   oracle_cc_bfs         plain definition, by BFS from each unlabelled
 *                         vertex in increasing id order (O2, independent)
 *   oracle_kout_sample    k-out sampling, Section 3.2 and Algorithm 4
 *   oracle_bfs_sample     BFS sampling, Section 3.2 and Algorithm 5
 *   oracle_ldd_sample     LDD sampling, Section 3.2, Algorithm 6, and the
 *                         mechanism of Appendix B.3 (exponential start
 *                         times, simultaneous BFS)
 *   oracle_identify_frequent   IdentifyFrequent of Algorithm 1
 *   oracle_finish_uf      union-find finish, Algorithm 7 (sequential)
 *   oracle_finish_sv      Shiloach-Vishkin finish, Algorithm 15 (rounds)
 *   oracle_finish_lt_prf  Liu-Tarjan PRF finish, Appendix D (rounds)
 *   oracle_connectivity   Algorithm 1 composed from the above
 *   oracle_incr_*         batch-incremental setting, Section 3.5 and
 *                         Appendix B.4 (inserts, then queries, per batch)
 *   oracle_spanning_forest   spanning forest (Section 3.5 "Spanning Forest"
 *                         and its appendix): the edges whose union joined
 *                         two trees in a sequential union-find (O1)
 *   oracle_check_forest   validity of any claimed spanning forest: every
 *                         pair is an edge of G, the pairs are acyclic, and
 *                         they connect exactly the components of G
 *   oracle_msf_kruskal    exact minimum spanning forest (plain definition,
 *                         by Kruskal's algorithm)
 *   oracle_amsf           approximate minimum spanning forest, Section 5.1:
 *                         weight buckets [Wmin(1+eps)^i, Wmin(1+eps)^(i+1)),
 *                         smallest first, a spanning forest of each bucket
 *                         over the labelling of the buckets before it
 *
 * Random draws: counter-based, the ctr-th output of a SplitMix64 sequence
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): out(s, ctr) = mix64(s + (ctr + 1) * 0x9E3779B97F4A7C15),
 * mix64 being that paper's finaliser.  Written here from its definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define NONE 0xFFFFFFFFu

/* ---- counter-based random draws (SplitMix64) ------------------------- */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
uint64_t oracle_draw(uint64_t seed, uint64_t ctr) {
    return mix64(seed + (ctr + 1) * 0x9E3779B97F4A7C15ull);
}
/* stream tags that separate the independent draws of one seed */
#define TAG_KOUT 0x6B6F7574ull   /* k-out neighbour picks   */
#define TAG_BFS  0x62667373ull   /* BFS sampling sources    */
#define TAG_FREQ 0x66726571ull   /* IdentifyFrequent sample */

/* ---- sequential union-find used by O1, k-out and the UF finish ------- */
static uint32_t uf_find(uint32_t *P, uint32_t x) {
    while (P[x] != x) {            /* path halving */
        P[x] = P[P[x]];
        x = P[x];
    }
    return x;
}
/* link the larger root under the smaller: keeps P[x] <= x, so every root is
 * the minimum of its tree.  Returns 1 if two trees were joined. */
static int uf_union(uint32_t *P, uint32_t u, uint32_t v) {
    uint32_t ru = uf_find(P, u), rv = uf_find(P, v);
    if (ru == rv) return 0;
    if (ru < rv) P[rv] = ru; else P[ru] = rv;
    return 1;
}

/* O1: label[v] = min id of v's component, by union-find over every edge. */
uint64_t oracle_cc_uf(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *label) {
    uint64_t links = 0;
    for (uint32_t i = 0; i < n; i++) label[i] = i;
    for (uint32_t u = 0; u < n; u++)
        for (uint64_t e = I[u]; e < I[u + 1]; e++) links += uf_union(label, u, A[e]);
    for (uint32_t v = 0; v < n; v++) label[v] = uf_find(label, v);
    return links;   /* = n - #components */
}

/* O1's union loop restricted to the edges of vertices [0, u_end), on a
 * caller-initialised forest P (identity for a fresh start): a bounded
 * slice of the same work, used to time the oracle on a sample of a large
 * graph.  Returns the number of edges processed. */
uint64_t oracle_uf_prefix(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t u_end, uint32_t *P) {
    uint64_t e_done = 0;
    if (u_end > n) u_end = n;
    for (uint32_t u = 0; u < u_end; u++) {
        for (uint64_t e = I[u]; e < I[u + 1]; e++) uf_union(P, u, A[e]);
        e_done += I[u + 1] - I[u];
    }
    return e_done;
}

/* O2: BFS from each unlabelled vertex in increasing id order; the source is
 * the smallest id of its component because every smaller vertex is already
 * labelled.  Shares nothing with O1. */
int oracle_cc_bfs(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *label) {
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!queue) return -1;
    for (uint32_t i = 0; i < n; i++) label[i] = NONE;
    for (uint32_t s = 0; s < n; s++) {
        if (label[s] != NONE) continue;
        uint32_t head = 0, tail = 0;
        label[s] = s;
        queue[tail++] = s;
        while (head < tail) {
            uint32_t x = queue[head++];
            for (uint64_t e = I[x]; e < I[x + 1]; e++) {
                uint32_t y = A[e];
                if (label[y] == NONE) { label[y] = s; queue[tail++] = y; }
            }
        }
    }
    free(queue);
    return 0;
}

/* ---- IdentifyFrequent (Algorithm 1) ----------------------------------- */
/* L_max = the most frequent label; ties go to the smallest label.  With
 * samples == 0 every label is counted; with samples > 0 only the labels at
 * the positions out(seed ^ TAG_FREQ, i) mod n, i < samples, are counted
 * (an estimate: L_max changes only the work of the finish, never its
 * result).  *count_out receives the winner's count in what was counted. */
uint32_t oracle_identify_frequent(uint32_t n, const uint32_t *label, uint32_t samples,
                                  uint64_t seed, uint64_t *count_out) {
    if (n == 0) { if (count_out) *count_out = 0; return NONE; }
    uint32_t *cnt = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!cnt) return NONE;
    if (samples == 0) {
        for (uint32_t v = 0; v < n; v++) cnt[label[v]]++;
    } else {
        for (uint32_t i = 0; i < samples; i++)
            cnt[label[oracle_draw(seed ^ TAG_FREQ, i) % n]]++;
    }
    uint32_t best = 0;
    for (uint32_t l = 1; l < n; l++)
        if (cnt[l] > cnt[best]) best = l;
    if (count_out) *count_out = cnt[best];
    free(cnt);
    return best;
}

/* ---- k-out sampling (Section 3.2, Algorithm 4; variants, Appendix C.4) - */
/* Neighbour pick j (0 <= j < k) of vertex v (deg > 0) under the selection
 * rule: 0 hybrid (the first edge, then k - 1 uniform picks), 1 afforest
 * (the first k edges; pick j exists only if j < deg), 2 pure (k uniform
 * picks).  A uniform pick is A[I[v] + r], r = floor(hi32(out(seed ^
 * TAG_KOUT, v*k + j)) * deg / 2^32), with replacement.  NONE: no pick. */
uint32_t oracle_kout_pick(const uint64_t *I, const uint32_t *A, uint32_t v, uint32_t k,
                          uint32_t j, uint64_t seed, int rule) {
    uint64_t deg = I[v + 1] - I[v];
    if (rule == 1) return j < deg ? A[I[v] + j] : NONE;
    if (rule == 0 && j == 0) return A[I[v]];
    uint64_t h = oracle_draw(seed ^ TAG_KOUT, (uint64_t)v * k + j) >> 32;
    return A[I[v] + ((h * deg) >> 32)];
}

/* Sampled labels: union-find over the picked edges, then full compression,
 * so label[v] = min id of v's component in the sampled subgraph. */
void oracle_kout_sample(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t k,
                        uint64_t seed, int rule, uint32_t *label) {
    for (uint32_t i = 0; i < n; i++) label[i] = i;
    for (uint32_t v = 0; v < n; v++) {
        if (I[v + 1] == I[v]) continue;
        for (uint32_t j = 0; j < k; j++) {
            uint32_t w = oracle_kout_pick(I, A, v, k, j, seed, rule);
            if (w != NONE) uf_union(label, v, w);
        }
    }
    for (uint32_t v = 0; v < n; v++) label[v] = uf_find(label, v);
}

/* ---- sampled clusters to min-id stars --------------------------------- */
/* BFS and LDD label a cluster by its source/centre, which need not be the
 * cluster's smallest member.  Each cluster is relabelled to its smallest
 * member (a depth-1 star under the minimum), the form a min-linking
 * union-find finish needs.  Pure relabelling: the partition is unchanged. */
static int relabel_to_min(uint32_t n, uint32_t *label) {
    uint32_t *cmin = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!cmin) return -1;
    for (uint32_t i = 0; i < n; i++) cmin[i] = NONE;
    for (uint32_t v = 0; v < n; v++) if (v < cmin[label[v]]) cmin[label[v]] = v;
    for (uint32_t v = 0; v < n; v++) label[v] = cmin[label[v]];
    free(cmin);
    return 0;
}

/* ---- BFS sampling (Section 3.2, Algorithm 5) -------------------------- */
/* For try i < tries: source s = out(seed ^ TAG_BFS, i) mod n; label[u] = s if
 * u is reachable from s, else u; stop if the most frequent label makes up
 * more than 10% of the labels (10 * count > n); after all tries fail the
 * identity labelling is returned.  The result is relabelled to min-id stars.
 * Returns the successful try's index, or -1. */
int oracle_bfs_sample(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t tries,
                      uint64_t seed, uint32_t *label) {
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    int found = -1;
    if (!queue) return -2;
    for (uint32_t i = 0; i < tries && n > 0; i++) {
        uint32_t s = (uint32_t)(oracle_draw(seed ^ TAG_BFS, i) % n);
        for (uint32_t v = 0; v < n; v++) label[v] = v;
        /* LabelSpreadingBFS: reachability from s (direction does not change it) */
        uint8_t *seen = (uint8_t *)calloc(n, 1);
        uint32_t head = 0, tail = 0;
        seen[s] = 1; queue[tail++] = s;
        while (head < tail) {
            uint32_t x = queue[head++];
            label[x] = s;
            for (uint64_t e = I[x]; e < I[x + 1]; e++)
                if (!seen[A[e]]) { seen[A[e]] = 1; queue[tail++] = A[e]; }
        }
        free(seen);
        uint64_t c = 0;
        oracle_identify_frequent(n, label, 0, 0, &c);
        if (10 * c > (uint64_t)n) { found = (int)i; break; }
    }
    if (found < 0) for (uint32_t v = 0; v < n; v++) label[v] = v;
    free(queue);
    relabel_to_min(n, label);
    return found;
}

/* ---- LDD sampling (Section 3.2, Algorithm 6, Appendix B.3) ------------ */
/* One round of Miller-Peng-Xu clustering with exponential start times and
 * no random permutation: vertices are started in id order, round r starting
 * the next floor(exp(beta * r)) ids (S_0 = 0, S_{r+1} = min(n, S_r +
 * floor(exp(beta r)))), so that the number started grows geometrically as
 * exponential shifts make it.  In round r, first every still-uncovered id in
 * [S_r, S_{r+1}) becomes the centre of its own cluster; then the frontier
 * (the vertices covered in round r-1 plus the new centres) claims every
 * uncovered neighbour, a vertex claimed by several clusters in one round
 * taking the smallest centre id.  Rounds run until every vertex is covered.
 * The clusters are returned relabelled to min-id stars.  Returns #rounds. */
uint64_t oracle_ldd_schedule(uint32_t n, double beta, uint32_t round) {
    (void)n;
    double x = floor(exp(beta * (double)round));
    if (x < 1.0) x = 1.0;
    if (x > 4294967295.0) x = 4294967295.0;
    return (uint64_t)x;
}
int oracle_ldd_sample(uint32_t n, const uint64_t *I, const uint32_t *A, double beta,
                      uint32_t *label) {
    uint32_t *front = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *next = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!front || !next || !cand) return -1;
    for (uint32_t v = 0; v < n; v++) { label[v] = NONE; cand[v] = NONE; }
    uint64_t S = 0, covered = 0;
    uint32_t nf = 0;
    int rounds = 0;
    while (covered < n) {
        uint64_t add = oracle_ldd_schedule(n, beta, (uint32_t)rounds);
        uint64_t S1 = S + add < n ? S + add : n;
        for (uint64_t v = S; v < S1; v++)
            if (label[v] == NONE) { label[v] = (uint32_t)v; front[nf++] = (uint32_t)v; covered++; }
        S = S1;
        /* one hop of the simultaneous BFS: candidates first, then commit */
        uint32_t nn = 0;
        for (uint32_t i = 0; i < nf; i++) {
            uint32_t x = front[i];
            for (uint64_t e = I[x]; e < I[x + 1]; e++) {
                uint32_t y = A[e];
                if (label[y] != NONE) continue;
                if (cand[y] == NONE) next[nn++] = y;
                if (label[x] < cand[y]) cand[y] = label[x];
            }
        }
        for (uint32_t i = 0; i < nn; i++) { label[next[i]] = cand[next[i]]; cand[next[i]] = NONE; }
        covered += nn;
        uint32_t *t = front; front = next; next = t;
        nf = nn;
        rounds++;
    }
    free(front); free(next); free(cand);
    relabel_to_min(n, label);
    return rounds;
}

/* ---- finish methods --------------------------------------------------- */
/* Union-find finish (Algorithm 7), sequential: for every u whose sampled
 * label differs from L_max, apply Union(u, v) to each edge (u, v).  Edges
 * out of L_max are skipped; they are applied from their other endpoint
 * because the graph is symmetric (Theorem B.2's argument).  label[] holds
 * sampled labels that form min-rooted stars; on return it holds the
 * canonical min-id labels.  Returns the number of edges applied. */
uint64_t oracle_finish_uf(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *label,
                          uint32_t lmax) {
    uint8_t *skip = (uint8_t *)malloc(n ? n : 1);
    uint64_t applied = 0;
    for (uint32_t u = 0; u < n; u++) skip[u] = (lmax != NONE && label[u] == lmax);
    for (uint32_t u = 0; u < n; u++) {
        if (skip[u]) continue;
        for (uint64_t e = I[u]; e < I[u + 1]; e++) { uf_union(label, u, A[e]); applied++; }
    }
    for (uint32_t v = 0; v < n; v++) label[v] = uf_find(label, v);
    free(skip);
    return applied;
}

/* FullShortcut: point every vertex straight at its root. */
static void full_shortcut(uint32_t n, uint32_t *P) {
    for (uint32_t v = 0; v < n; v++) {
        uint32_t r = v;
        while (P[r] != r) r = P[r];
        P[v] = r;
    }
}

/* Shiloach-Vishkin finish (Algorithm 15): rounds of (i) for each candidate
 * vertex u (sampled label != L_max) and edge (u, v): l = min(P[u], P[v]),
 * h = max(...); if l != h and h was a root at the start of the round, hook
 * h under l with writeMin and note a change; (ii) FullShortcut, and the
 * round-start snapshot is refreshed.  Until a round notes no change.
 * Returns the number of rounds. */
int oracle_finish_sv(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *P, uint32_t lmax) {
    uint8_t *cand = (uint8_t *)malloc(n ? n : 1);
    uint32_t *prev = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    int rounds = 0, changed = 1;
    for (uint32_t u = 0; u < n; u++) { cand[u] = !(lmax != NONE && P[u] == lmax); prev[u] = P[u]; }
    while (changed) {
        changed = 0;
        for (uint32_t u = 0; u < n; u++) {
            if (!cand[u]) continue;
            for (uint64_t e = I[u]; e < I[u + 1]; e++) {
                uint32_t pu = P[u], pv = P[A[e]];
                uint32_t l = pu < pv ? pu : pv, h = pu < pv ? pv : pu;
                if (l != h && prev[h] == h) {
                    if (l < P[h]) P[h] = l;   /* writeMin */
                    changed = 1;
                }
            }
        }
        full_shortcut(n, P);
        memcpy(prev, P, sizeof(uint32_t) * n);
        rounds++;
    }
    free(cand); free(prev);
    return rounds;
}

/* Liu-Tarjan PRF finish (Appendix D: ParentConnect, RootUpdate,
 * FullShortcut): rounds of (i) for each candidate u and edge (u, v), the
 * parents of both endpoints are candidates for each other: x = P[u] takes
 * y = P[v] if y < P[x] and x was a root at the start of the round, and
 * symmetrically; (ii) FullShortcut.  Until the parent array stops changing.
 * Returns the number of rounds. */
int oracle_finish_lt_prf(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *P, uint32_t lmax) {
    uint8_t *cand = (uint8_t *)malloc(n ? n : 1);
    uint32_t *prev = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    int rounds = 0, changed = 1;
    for (uint32_t u = 0; u < n; u++) { cand[u] = !(lmax != NONE && P[u] == lmax); prev[u] = P[u]; }
    while (changed) {
        changed = 0;
        for (uint32_t u = 0; u < n; u++) {
            if (!cand[u]) continue;
            for (uint64_t e = I[u]; e < I[u + 1]; e++) {
                uint32_t x = P[u], y = P[A[e]];
                if (y < P[x] && prev[x] == x) { P[x] = y; changed = 1; }
                if (x < P[y] && prev[y] == y) { P[y] = x; changed = 1; }
            }
        }
        full_shortcut(n, P);
        for (uint32_t v = 0; v < n; v++) { if (prev[v] != P[v]) changed = 1; prev[v] = P[v]; }
        rounds++;
    }
    free(cand); free(prev);
    return rounds;
}

/* ---- Algorithm 1 ------------------------------------------------------ */
/* sample: 0 none, 1 k-out (kout_rule: 0 hybrid, 1 afforest, 2 pure), 2 BFS,
 * 3 LDD; finish: 0/1 union-find (all
 * union-find variants reach the same sequential result), 2 SV, 3 LT-PRF.
 * With no sampling there is no frequent component to skip.
 * stats (optional, 4 entries): L_max, edges applied by a union-find finish
 * (0 otherwise), rounds of an SV/LT finish (0 otherwise), sampling result
 * (BFS try index or LDD rounds). */
int oracle_connectivity(uint32_t n, const uint64_t *I, const uint32_t *A, int sample, uint32_t k,
                        int kout_rule, uint32_t tries, double beta, uint64_t seed, uint32_t freq_samples,
                        int finish, uint32_t *label, uint64_t *stats) {
    uint64_t st[4] = {NONE, 0, 0, 0};
    for (uint32_t i = 0; i < n; i++) label[i] = i;
    switch (sample) {
        case 0: break;
        case 1: oracle_kout_sample(n, I, A, k, seed, kout_rule, label); break;
        case 2: st[3] = (uint64_t)(int64_t)oracle_bfs_sample(n, I, A, tries, seed, label); break;
        case 3: st[3] = (uint64_t)oracle_ldd_sample(n, I, A, beta, label); break;
        default: return -1;
    }
    uint32_t lmax = NONE;
    if (sample != 0) lmax = oracle_identify_frequent(n, label, freq_samples, seed, NULL);
    st[0] = lmax;
    switch (finish) {
        case 0: case 1: st[1] = oracle_finish_uf(n, I, A, label, lmax); break;
        case 2: st[2] = (uint64_t)oracle_finish_sv(n, I, A, label, lmax); break;
        case 3: st[2] = (uint64_t)oracle_finish_lt_prf(n, I, A, label, lmax); break;
        default: return -1;
    }
    if (stats) memcpy(stats, st, sizeof(st));
    return 0;
}

/* ---- batch-incremental connectivity (Section 3.5, Appendix B.4) ------- */
/* A batch's inserts are applied first, then its queries are answered
 * (phase-concurrent semantics): a query sees every insert of its own and of
 * earlier batches.  The state is the union-find forest of O1. */
void oracle_incr_insert(uint32_t n, uint32_t *P, const uint32_t *pairs, uint64_t k) {
    (void)n;
    for (uint64_t i = 0; i < k; i++) uf_union(P, pairs[2 * i], pairs[2 * i + 1]);
}
void oracle_incr_query(uint32_t n, uint32_t *P, const uint32_t *pairs, uint64_t q, uint8_t *ans) {
    (void)n;
    for (uint64_t i = 0; i < q; i++) ans[i] = uf_find(P, pairs[2 * i]) == uf_find(P, pairs[2 * i + 1]);
}
void oracle_incr_labels(uint32_t n, uint32_t *P, uint32_t *label) {
    for (uint32_t v = 0; v < n; v++) label[v] = uf_find(P, v);
}

/* ---- spanning forest -------------------------------------------------- */
/* A spanning forest of G: one tree per component, n - #components edges.
 * Sequential union-find over every edge; an edge is kept iff its union
 * joined two different trees.  Returns the number of pairs written to
 * out[2*i], out[2*i+1] (room for 2*(n-1) words). */
uint64_t oracle_spanning_forest(uint32_t n, const uint64_t *I, const uint32_t *A, uint32_t *out) {
    uint32_t *P = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    uint64_t cnt = 0;
    for (uint32_t v = 0; v < n; ++v) P[v] = v;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = I[u]; e < I[u + 1]; ++e)
            if (uf_union(P, u, A[e])) {
                out[2 * cnt] = u;
                out[2 * cnt + 1] = A[e];
                ++cnt;
            }
    free(P);
    return cnt;
}

/* is (u, v) an edge of G?  adjacency lists sorted: binary search, else scan */
static int has_edge(const uint64_t *I, const uint32_t *A, uint32_t u, uint32_t v, int sorted) {
    uint64_t lo = I[u], hi = I[u + 1];
    if (!sorted) {
        for (uint64_t e = lo; e < hi; ++e)
            if (A[e] == v) return 1;
        return 0;
    }
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (A[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < I[u + 1] && A[lo] == v;
}

/* Checks a claimed spanning forest F (count pairs) of G against the
 * canonical labels `label` of G.  Returns 0 if F is a spanning forest, else
 * the first failed property: 1 a pair with an endpoint >= n, 2 a pair that
 * is not an edge of G, 3 a pair that closes a cycle in F, 4 a pair joining
 * two different components of G, 5 F's components differ from G's (too few
 * pairs). */
int oracle_check_forest(uint32_t n, const uint64_t *I, const uint32_t *A, const uint32_t *pairs, uint64_t count,
                        const uint32_t *label) {
    int sorted = 1;
    for (uint32_t u = 0; u < n && sorted; ++u)
        for (uint64_t e = I[u] + 1; e < I[u + 1]; ++e)
            if (A[e - 1] > A[e]) { sorted = 0; break; }
    uint32_t *P = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) P[v] = v;
    int bad = 0;
    for (uint64_t i = 0; i < count && !bad; ++i) {
        uint32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        if (u >= n || v >= n) bad = 1;
        else if (!has_edge(I, A, u, v, sorted)) bad = 2;
        else if (label[u] != label[v]) bad = 4;
        else if (!uf_union(P, u, v)) bad = 3;
    }
    if (!bad) {
        /* acyclic pairs inside G's components: F spans them iff it has
         * exactly n - #components pairs */
        uint64_t comps = 0;
        for (uint32_t v = 0; v < n; ++v) comps += label[v] == v;
        if (count != (uint64_t)n - comps) bad = 5;
    }
    free(P);
    return bad;
}

/* ---- minimum spanning forests ---------------------------------------- */
/* Undirected edges (u < v) of a symmetric weighted CSR, as indices into A. */
static uint64_t upper_edges(uint32_t n, const uint64_t *I, const uint32_t *A, uint64_t *idx, uint32_t *src) {
    uint64_t k = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = I[u]; e < I[u + 1]; ++e)
            if (A[e] > u) { idx[k] = e; src[k] = u; ++k; }
    return k;
}

static const float *g_w;   /* weights seen by the comparator */
static int by_weight(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    if (g_w[x] < g_w[y]) return -1;
    if (g_w[x] > g_w[y]) return 1;
    return x < y ? -1 : (x > y);
}

/* Exact MSF: Kruskal over the undirected edges sorted by weight (ties by
 * CSR position).  Writes the forest pairs, returns their number, and the
 * total weight (summed in double) in *weight. */
uint64_t oracle_msf_kruskal(uint32_t n, const uint64_t *I, const uint32_t *A, const float *W, uint32_t *out,
                            double *weight) {
    uint64_t m = I[n];
    uint64_t *idx = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    uint32_t *src = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *owner = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t k = upper_edges(n, I, A, idx, src);
    for (uint64_t i = 0; i < k; ++i) owner[idx[i]] = src[i];
    g_w = W;
    qsort(idx, k, sizeof(uint64_t), by_weight);
    uint32_t *P = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) P[v] = v;
    uint64_t cnt = 0;
    double total = 0.0;
    for (uint64_t i = 0; i < k; ++i) {
        uint64_t e = idx[i];
        uint32_t u = owner[e], v = A[e];
        if (uf_union(P, u, v)) {
            out[2 * cnt] = u;
            out[2 * cnt + 1] = v;
            ++cnt;
            total += W[e];
        }
    }
    free(P);
    free(owner);
    free(src);
    free(idx);
    *weight = total;
    return cnt;
}

/* Bucket of weight w: floor(log(w / Wmin) / log(1 + eps)), clamped at 0. */
static uint64_t weight_bucket(float w, float wmin, double eps) {
    double b = floor(log((double)w / (double)wmin) / log1p(eps));
    return b < 0.0 ? 0u : (uint64_t)b;
}

/* Approximate MSF (the folklore bucketed algorithm of Section 5.1): buckets
 * in increasing weight order; within a bucket every edge whose endpoints
 * are not yet connected joins the forest (a spanning forest of the bucket's
 * edges over the labelling so far).  Sequential, no skipping.  Empty
 * buckets do nothing, so the edges are visited sorted by (bucket, CSR
 * position): the bucket order, and vertex order inside a bucket. */
static const uint64_t *g_bucket;
static int by_bucket(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    if (g_bucket[x] != g_bucket[y]) return g_bucket[x] < g_bucket[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}

uint64_t oracle_amsf(uint32_t n, const uint64_t *I, const uint32_t *A, const float *W, double eps, uint32_t *out,
                     double *weight) {
    uint64_t m = I[n];
    float wmin = 0.0f;
    for (uint64_t e = 0; e < m; ++e)
        if (e == 0 || W[e] < wmin) wmin = W[e];
    uint64_t *bucket = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    uint32_t *owner = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t *order = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = I[u]; e < I[u + 1]; ++e) owner[e] = u;
    for (uint64_t e = 0; e < m; ++e) {
        bucket[e] = weight_bucket(W[e], wmin, eps);
        order[e] = e;
    }
    g_bucket = bucket;
    qsort(order, m, sizeof(uint64_t), by_bucket);
    uint32_t *P = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) P[v] = v;
    uint64_t cnt = 0;
    double total = 0.0;
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t e = order[i];
        if (uf_union(P, owner[e], A[e])) {
            out[2 * cnt] = owner[e];
            out[2 * cnt + 1] = A[e];
            ++cnt;
            total += W[e];
        }
    }
    free(P);
    free(order);
    free(owner);
    free(bucket);
    *weight = total;
    return cnt;
}
