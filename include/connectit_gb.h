/*
 * connectit_gb.h -- C ABI of a GB300 (sm_103a) implementation of ConnectIt's
 * static and incremental graph connectivity (Dhulipala, Hong, Shun,
 * "ConnectIt: A Framework for Static and Incremental Parallel Graph
 * Connectivity Algorithms").
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Graph: symmetric CSR (Section 2, "Graph Notation and Formats").  `offsets`
 *   holds n+1 entries (uint32 when offsets_u64 == 0, else uint64) with
 *   offsets[0] = 0 and offsets[n] = m; `edges` holds m uint32 vertex ids; the
 *   neighbours of v are edges[offsets[v] .. offsets[v+1]-1].  Every
 *   undirected edge must be stored in both directions (the finish methods
 *   skip the edges out of the largest sampled component and rely on the
 *   reverse copy, Theorem B.2).  Self-loops and duplicates are allowed.
 * Result: canonical labels, labels[v] = the smallest vertex id of v's
 *   connected component (a connectivity labelling, Section 2, in the unique
 *   min-id form).  Every sampling x finish combination writes the same array.
 * Alignment: every array must be aligned to its element size (uint64 to 8,
 *   uint32 to 4 bytes); a misaligned pointer returns CC_ERR_INVALID.  Any
 *   sub-slice of an array is fine; wider vector accesses are used only where
 *   the library has checked the address.
 * Memory: every array argument is a DEVICE pointer owned by the caller,
 *   except in cc_static_host, whose arrays are host pointers.  The library
 *   allocates only its own scratch (stream-ordered, cudaMallocAsync on the
 *   call's stream) and frees it before the call's work completes.
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Work is enqueued on it.  Calls return once their work is enqueued, except
 *   where a method's loop depends on device data (BFS and LDD sampling, the
 *   SV and LT finishes), where the call waits on the stream between rounds.
 * Errors: argument checks are synchronous and return CC_ERR_INVALID before
 *   anything is enqueued.  Input faults found on the device (an edge id >= n,
 *   decreasing or out-of-range offsets) and iteration caps reached in a
 *   device loop never trap: kernels skip the bad access, record a bit in a
 *   per-device sticky error word and return.  cc_device_error() reads and
 *   clears that word; calls that synchronise anyway (cc_static_ex with
 *   stats, cc_static_host) return it as their status.
 * Threads: entry points may be called from several host threads on
 *   different streams; they share the sticky error word.
 */
#ifndef CONNECTIT_GB_H
#define CONNECTIT_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cc_status {
    CC_OK = 0,
    CC_ERR_INVALID = 1,        /* bad argument: nothing was enqueued */
    CC_ERR_OOM = 2,            /* scratch allocation failed */
    CC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    CC_ERR_NONCONVERGED = 4,   /* a device loop reached its iteration/time cap */
    CC_ERR_BAD_INPUT = 5,      /* device found an edge id >= n or bad offsets */
    CC_ERR_UNSUPPORTED = 6     /* option combination not provided */
} cc_status;

/* Device sticky-error bits (cc_device_error). */
#define CC_DEVERR_BAD_EDGE     1u
#define CC_DEVERR_BAD_OFFSETS  2u
#define CC_DEVERR_NONCONVERGED 4u

/* Sampling methods (Section 3.2; Algorithms 4-6). */
enum { CC_SAMPLE_NONE = 0, CC_SAMPLE_KOUT = 1, CC_SAMPLE_BFS = 2, CC_SAMPLE_LDD = 3 };
/* Finish methods (Section 3.3): UF-Rem-CAS (Algorithm 14), UF-Async
 * (Algorithm 10), Shiloach-Vishkin (Algorithm 15), Liu-Tarjan PRF
 * (ParentConnect + RootUpdate + FullShortcut, Appendix D). */
enum { CC_FINISH_UF_REM_CAS = 0, CC_FINISH_UF_ASYNC = 1, CC_FINISH_SV = 2, CC_FINISH_LT_PRF = 3,
       CC_FINISH_UF_HOOKS = 4, CC_FINISH_UF_EARLY = 5, CC_FINISH_LIU_TARJAN = 6, CC_FINISH_STERGIOU = 7,
       CC_FINISH_LABEL_PROP = 8 };
/* Liu-Tarjan rules (CC_FINISH_LIU_TARJAN, field lt_rules; Section 3.3 and
 * the appendix's list of sixteen variants): connect = CONNECT, PARENT or
 * EXTENDED, plus ROOTUP (RootUpdate), FULL (FullShortcut instead of one
 * Shortcut step) and ALTER.  Valid: CONNECT with ALTER (CUSA, CRSA, CUFA,
 * CRFA); PARENT with anything (PUSA, PRSA, PUS, PRS, PUFA, PRFA, PUF, PRF);
 * EXTENDED without ROOTUP (EUSA, EUS, EUFA, EUF).  CC_FINISH_LT_PRF is the
 * root-based PRF with its own kernels. */
enum { CC_LT_CONNECT = 0, CC_LT_PARENT = 1, CC_LT_EXTENDED = 2, CC_LT_ROOTUP = 4, CC_LT_FULL = 8,
       CC_LT_ALTER = 16 };
/* Find options (Algorithm 8): no compaction, atomic path splitting, atomic
 * path halving, full compression of the find path.  For UF-Rem-CAS this is
 * the Compress option of Algorithm 14, which excludes FindCompress. */
enum { CC_FIND_NAIVE = 0, CC_FIND_SPLIT = 1, CC_FIND_HALVE = 2, CC_FIND_COMPRESS = 3 };
/* Splice options of Rem's algorithm (Algorithm 9).  SpliceAtomic is correct
 * phase-concurrently (every call here separates unions from finds) and is
 * not root-based, so cc_spanning_forest rejects it. */
enum { CC_SPLICE_SPLIT_ONE = 0, CC_SPLICE_HALVE_ONE = 1, CC_SPLICE_ATOMIC = 2 };
/* k-out selection rules (Appendix C.4): hybrid, the first edge and k - 1
 * uniform picks; afforest, the first k edges; pure, k uniform picks. */
enum { CC_KOUT_HYBRID = 0, CC_KOUT_AFFOREST = 1, CC_KOUT_PURE = 2 };

typedef struct cc_sample_opt {
    int32_t kind;          /* CC_SAMPLE_* */
    uint32_t k;            /* k-out: edges per vertex (1..64; 2) */
    uint32_t bfs_tries;    /* BFS: number of tries c (>= 1; 3) */
    float ldd_beta;        /* LDD: beta in (0, 64] (0.2) */
    uint64_t seed;         /* seed of every random draw (k-out picks, BFS sources, freq sample) */
    uint32_t freq_samples; /* IdentifyFrequent: 0 counts all n labels; S in [1, 4096] counts S
                              seeded sample positions (an estimate; changes work, not labels) */
    uint32_t kout_rule;    /* k-out: CC_KOUT_* (CC_KOUT_HYBRID) */
} cc_sample_opt;

typedef struct cc_finish_opt {
    int32_t kind;          /* CC_FINISH_* */
    int32_t find;          /* CC_FIND_* (union-find finishes) */
    int32_t splice;        /* CC_SPLICE_* (UF-Rem-CAS) */
    int32_t lt_rules;      /* CC_LT_* bits (CC_FINISH_LIU_TARJAN); 0 for every other kind */
} cc_finish_opt;

/* Counters of one cc_static_ex call. */
typedef struct cc_stats {
    uint32_t lmax;          /* L_max, the frequent sampled label (0xFFFFFFFF with no sampling) */
    int32_t sample_info;    /* BFS: index of the successful try or -1; LDD: rounds; else 0 */
    uint32_t rounds;        /* SV / LT: rounds run; union-find: 0 */
    uint32_t reserved;
    uint64_t edges_finish;  /* directed edges read by the finish (out of non-L_max vertices) */
} cc_stats;

/* Sensible defaults: k-out k=2, c=3 BFS tries, LDD beta=0.2, seed 1, exact
 * IdentifyFrequent; UF-Rem-CAS with SplitAtomicOne and no extra compression. */
void cc_default_opts(cc_sample_opt *sample, cc_finish_opt *finish);

/* Static connectivity, Algorithm 1: labels <- identity; SampleComponents;
 * L_max <- IdentifyFrequent; FinishComponents skipping the vertices whose
 * sampled label is L_max; then a final shortcut to canonical min-id labels.
 * labels_out: device uint32[n], written (it also serves as the parent array
 * during the call).  sample/finish: host pointers; NULL = defaults. */
cc_status cc_static(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                    uint64_t m, const cc_sample_opt *sample, const cc_finish_opt *finish,
                    uint32_t *labels_out, void *stream);

/* cc_static plus counters: when stats != NULL the call synchronises the
 * stream, fills *stats (host memory) and returns the device error status. */
cc_status cc_static_ex(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                       uint64_t m, const cc_sample_opt *sample, const cc_finish_opt *finish,
                       uint32_t *labels_out, cc_stats *stats, void *stream);

/* Spanning forest (Section 3.5 "Spanning Forest" and the spanning-forest
 * algorithm of its appendix): the same sampling / IdentifyFrequent / finish
 * pipeline, where the sampling emits its tree edges (k-out: each edge that
 * hooked a root; BFS: the tree edge at each child; LDD: the searches' tree
 * edges) and the root-based finish stores each edge that hooked a root; the
 * non-empty slots are then filtered into forest_out.
 * forest_out: device uint32[2*n] (room for n pairs), receives *count_out
 *   pairs (u, v), each an edge of G, in no particular order; the pairs form
 *   a forest whose trees span exactly the components of G, so
 *   *count_out = n - #components.  Which spanning forest is returned depends
 *   on thread timing; its size and the components it spans do not.
 * count_out: host uint64, written before the call returns (it synchronises
 *   the stream).
 * labels_out: optional device uint32[n], the canonical labels (NULL: not
 *   returned; scratch is used instead).
 * Finishes: the root-based union-find finishes (UF-Rem-CAS without
 * SpliceAtomic, UF-Async, UF-Hooks, UF-Early).  SV and LT-PRF return
 * CC_ERR_UNSUPPORTED (their writeMin hooks do not identify the winning edge
 * without another pass), as does SpliceAtomic (not root-based).  Returns
 * the device error status. */
cc_status cc_spanning_forest(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                             uint64_t m, const cc_sample_opt *sample, const cc_finish_opt *finish,
                             uint32_t *forest_out, uint64_t *count_out, uint32_t *labels_out, void *stream);

/* Approximate minimum spanning forest (Section 5.1): edge weights are
 * bucketed by ratio 1 + epsilon from the smallest weight, buckets are taken
 * lightest first, and each adds a spanning forest of its edges over the
 * connectivity of the lighter buckets (UF-Rem-CAS, SplitAtomicOne,
 * FindNaive).  The forest weighs at most (1 + epsilon) times a minimum
 * spanning forest (up to float rounding of the bucket bounds, about 1e-7
 * relative).
 * weights: device float[m], positive and finite, equal on both stored
 *   copies of an edge (other weights are skipped and flagged
 *   CC_DEVERR_BAD_EDGE).
 * epsilon in [1e-3, 64]; more than CC_AMSF_MAX_BUCKETS buckets between the
 *   smallest and largest weight: CC_ERR_INVALID.
 * mode: CC_AMSF_NF (every bucket reads the whole CSR), CC_AMSF_NF_S (the
 *   same, skipping the vertices of the largest component so far),
 *   CC_AMSF_COO (edges grouped by bucket first, each read once).
 * forest_out: device uint32[2*n] (room for n pairs), *count_out pairs;
 *   *weight_out: their total weight (host double).  labels_out: optional
 *   device uint32[n], canonical labels.  Synchronises the stream; returns
 *   the device error status. */
#define CC_AMSF_MAX_BUCKETS 65536
enum { CC_AMSF_NF = 0, CC_AMSF_NF_S = 1, CC_AMSF_COO = 2 };
cc_status cc_amsf(const void *offsets, int offsets_u64, const uint32_t *edges, const float *weights, uint32_t n,
                  uint64_t m, float epsilon, int mode, uint32_t *forest_out, uint64_t *count_out,
                  double *weight_out, uint32_t *labels_out, void *stream);

/* cc_static on HOST buffers (offsets, edges, labels_out in host memory,
 * ideally pinned): runs cc_static, copies the labels back and synchronises.
 * The graph is copied to library-allocated device memory first, except
 * with k-out sampling on pinned (device-addressable) offsets and edges:
 * then the sampling reads them in place (the offsets and about two 32-byte
 * sectors per vertex cross the host link instead of the whole CSR), and the
 * finish reads in place too when the frequent cluster holds at least a
 * quarter of the vertices (else the CSR is copied before the finish).
 * Returns the device error status. */
cc_status cc_static_host(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                         uint64_t m, const cc_sample_opt *sample, const cc_finish_opt *finish,
                         uint32_t *labels_out, void *stream);

/* The three phases of Algorithm 1 on their own (the same kernels cc_static
 * runs), so that each can be checked and timed alone.
 * cc_sample: labels <- identity, then SampleComponents (k-out: union-find
 *   over the picked edges and full compression; BFS / LDD: clusters), each
 *   sampled cluster relabelled to its smallest member (a min-rooted star).
 *   labels_out: device uint32[n].  *sample_info_out (host, may be NULL) gets
 *   the BFS try index / LDD rounds; it forces a synchronisation.
 * cc_identify_frequent: *lmax_out (DEVICE uint32) <- the most frequent
 *   label of labels[0..n) (ties: smallest label); freq_samples/seed as in
 *   cc_sample_opt.
 * cc_finish: labels_inout holds sampled labels (min-rooted stars, as
 *   cc_sample writes them); runs the finish skipping vertices whose label
 *   equals lmax (0xFFFFFFFF: skip none) and writes canonical labels. */
cc_status cc_sample(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                    uint64_t m, const cc_sample_opt *sample, uint32_t *labels_out,
                    int32_t *sample_info_out, void *stream);
cc_status cc_identify_frequent(const uint32_t *labels, uint32_t n, uint32_t freq_samples,
                               uint64_t seed, uint32_t *lmax_out, void *stream);
cc_status cc_finish(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                    uint64_t m, const cc_finish_opt *finish, uint32_t lmax, uint32_t *labels_inout,
                    uint32_t *rounds_out, void *stream);

/* IdentifyFrequent without allocating (no counterpart in the paper: it is
 * for callers that cannot allocate device memory where they need L_max,
 * e.g. a latency-critical serving loop where cudaMalloc / cudaFree would
 * synchronise the device, a host callback where allocation calls are not
 * allowed, or a process whose device memory another allocator owns).
 * Same result as cc_identify_frequent with freq_samples = 0: *lmax_out
 * (DEVICE uint32) <- the most frequent label of labels[0..n), ties to the
 * smallest (0xFFFFFFFF when n == 0).  Its count scratch is a fixed
 * file-scope device array of CC_NOALLOC_MAX_LABELS uint32 (16 MiB plus one
 * word), reserved on every GPU that loads the library until the process
 * exits.  n > CC_NOALLOC_MAX_LABELS returns CC_ERR_INVALID before anything
 * is enqueued.  Every call looks up the scratch's device address in the
 * current device's context (so a context created again after
 * cudaDeviceReset is served at its new address); the first call on a
 * device also loads the library's device code there, so make that first
 * call before any stream capture.  Every call reuses the same
 * scratch and zeroes the part it needs first, so calls whose work could
 * overlap on the GPU (unordered streams) race and must not be issued.
 * Label ids >= n are skipped and flagged (CC_DEVERR_BAD_EDGE). */
#define CC_NOALLOC_MAX_LABELS (1u << 22)
cc_status cc_identify_frequent_noalloc(const uint32_t *labels, uint32_t n, uint32_t *lmax_out, void *stream);

/* MapEdges and GatherEdges (Section 4, Table 8): per-vertex reductions over
 * the incident edges, the paper's floors for reading a graph and for one
 * indirect read per edge.  out (DEVICE uint32[n]): MapEdges writes the
 * number of edges it read (the degree); GatherEdges writes the sum, mod
 * 2^32, of x[w] over the neighbours w (x: DEVICE uint32[n]).  Edge ids >= n
 * are skipped and flagged. */
cc_status cc_map_edges(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                       uint32_t *out, void *stream);
cc_status cc_gather_edges(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                          const uint32_t *x, uint32_t *out, void *stream);

/* Random-sector read rate: for i < count, read word
 * floor(draw64(seed, i) * words / 2^64) of the device array x (uint32_t[words]),
 * where draw64 is SplitMix64 (Steele, Lea and Flood, 2014):
 * z = seed + (i + 1) * 0x9E3779B97F4A7C15, then the stafford-13 finaliser.
 * *out (one device uint32) = the sum of the words read, mod 2^32.  Each read
 * is one 32-byte sector at an unrelated position: on an array larger than
 * L2 it measures the device's rate for the access a k-out pick makes (one
 * random sector of the edge array), the ceiling of that sampling kernel.
 * Errors: CC_ERR_INVALID for a null or unaligned pointer, or words == 0
 * with count > 0.  Stream-ordered; *out is zeroed first on the stream. */
cc_status cc_random_sectors(const uint32_t *x, uint64_t words, uint64_t count, uint64_t seed, uint32_t *out,
                            void *stream);

/* Batched static connectivity of many independent graphs in one persistent
 * launch (no counterpart in the paper, which labels one graph per call).
 * Each graph is labelled as Algorithm 1 with no sampling would label it:
 * union-find finish (Rem's CAS rule, Algorithm 14) and final shortcut.
 * Packing: G graphs; gv (DEVICE uint64[G+1], gv[0] = 0, non-decreasing,
 *   gv[G] = V) gives graph g the packed vertices [gv[g], gv[g+1]).
 *   offsets (DEVICE, V+1 entries, uint32 or uint64 per offsets_u64) is one
 *   packed CSR: local vertex i of graph g has its neighbours at
 *   edges[offsets[gv[g]+i] .. offsets[gv[g]+i+1]), stored as LOCAL ids in
 *   [0, n_g).  M = total directed edges.  Every graph must be symmetric.
 * labels_out (DEVICE uint32[V]): local vertex i of graph g gets the smallest
 *   local id of its component.
 * opt: schedule; NULL = cc_batch_default_opt (1024 threads, 65536,
 *   mode 2).  threads per CTA in {128, 256, 512, 1024}; graphs of at most
 *   smem_max_vertices vertices (<= 65536) keep their parent array in shared
 *   memory as 16-bit local ids (2 bytes per vertex of the threshold per
 *   CTA), larger ones in their slice of labels_out; vertex_mode 0 = one
 *   thread per vertex, 1 = one warp per vertex, 2 = 32 vertices per warp,
 *   the warp walking their concatenated edge lists, 3 = mode 2 at two
 *   1024-thread CTAs per SM (threads must be 1024).  Graphs are taken
 *   largest first.  Any schedule gives the same labels.  Scratch: 4 G + 4
 *   bytes (stream-ordered).
 * cc_batched_autotune times every candidate schedule on this batch (it
 *   synchronises), writes the fastest to *best_out (host) and its time in
 *   ms to *best_ms_out (host, may be NULL), and leaves labels_out computed. */
typedef struct cc_batch_opt {
    uint32_t threads;
    uint32_t smem_max_vertices;
    uint32_t vertex_mode;
    uint32_t reserved;      /* must be 0 */
} cc_batch_opt;
void cc_batch_default_opt(cc_batch_opt *opt);
cc_status cc_batched(const uint64_t *gv, uint32_t G, const void *offsets, int offsets_u64, const uint32_t *edges,
                     uint64_t V, uint64_t M, const cc_batch_opt *opt, uint32_t *labels_out, void *stream);
cc_status cc_batched_autotune(const uint64_t *gv, uint32_t G, const void *offsets, int offsets_u64,
                              const uint32_t *edges, uint64_t V, uint64_t M, uint32_t *labels_out,
                              cc_batch_opt *best_out, float *best_ms_out, void *stream);

/* Batch-incremental connectivity (Section 3.5, Algorithm 3; Appendix B.4).
 * A handle owns a resident parent array P (n uint32 in device memory).
 * cc_incr_create runs Initialize: static connectivity of the base graph
 *   (offsets/edges device pointers; both may be NULL when m == 0) into P.
 *   Finish kinds: the union-find ones (Section 3.5's types 1 and 3) and SV
 *   / Liu-Tarjan PRF (type 2); the Liu-Tarjan rule sets, Stergiou and
 *   label propagation return CC_ERR_UNSUPPORTED.
 * cc_incr_insert_batch: Insert(u, v) for k pairs (device uint32[2k],
 *   interleaved u0 v0 u1 v1 ...), each a Union; with SV / PRF the batch's
 *   pairs go through that finish's rounds (hooks, full shortcut) until a
 *   round changes nothing, and the call synchronises once per round.
 * cc_incr_query_batch: IsConnected(u, v) for q pairs -> answers_out (device
 *   uint8[q], 1 = connected).  A query sees every insert enqueued earlier on
 *   the handle (inserts and queries are separate phases, the
 *   phase-concurrent setting of Section 3.5, type 3).
 * cc_incr_labels: canonical min-id labels of the current graph.
 * Pairs with an id >= n are skipped and flagged (CC_DEVERR_BAD_EDGE); their
 *   answers are 0.  Calls on one handle must be stream-ordered. */
typedef struct cc_incr cc_incr;
cc_status cc_incr_create(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                         uint64_t m, const cc_sample_opt *sample, const cc_finish_opt *finish,
                         void *stream, cc_incr **out);
cc_status cc_incr_insert_batch(cc_incr *h, const uint32_t *pairs, uint64_t k, void *stream);
cc_status cc_incr_query_batch(cc_incr *h, const uint32_t *pairs, uint64_t q, uint8_t *answers_out,
                              void *stream);
cc_status cc_incr_labels(cc_incr *h, uint32_t *labels_out, void *stream);
uint32_t cc_incr_num_vertices(const cc_incr *h);
cc_status cc_incr_destroy(cc_incr *h);

/* Continuous-batching request loop over an incremental handle (no
 * counterpart in the paper; it serves Section 3.5's batch semantics to many
 * clients).  Requests are linearised in ticket order: request r's inserts are
 * applied, then its queries answered, after every request with a smaller
 * ticket, so each answer is the same alone or in the mix.  A dispatcher
 * thread admits requests as device slots free up (slots x slot_pairs pairs
 * of device memory, 9 bytes per pair; larger requests are split into
 * chunks, inserts first) and overlaps one request's copies with another's
 * kernels on separate streams.
 * cc_server_create: the server uses `h` exclusively until it is destroyed.
 * cc_server_submit: inserts (2k uint32) and queries (2q uint32) are HOST
 *   arrays, answers a HOST uint8[q] array; all three must stay valid until
 *   cc_server_wait returns.  A request whose three arrays are all pinned
 *   (device-mapped) host memory is read and written in place by the
 *   kernels (no copy, no slot); other requests are staged through the
 *   slots, the copy engines moving request r+1's pairs in while request
 *   r's kernels run.  With CC_SERVER_STAGE in flags every request is staged
 *   (measured slower for pinned requests on Grace-Blackwell: 6.2e9 against
 *   1.45e10 operations/s on the 1,000-batch workload at 90% queries).
 * cc_server_wait: blocks until the request's answers are in host memory;
 *   *latency_ms_out (may be NULL) gets submit-to-completion time.
 * cc_server_destroy: drains the queue, then frees the server (not h). */
typedef struct cc_server cc_server;
#define CC_SERVER_STAGE 1u
typedef struct cc_server_opt {
    uint32_t slots;        /* device slots in flight (1..64; 4) */
    uint32_t flags;        /* 0 or CC_SERVER_STAGE (default 0) */
    uint64_t slot_pairs;   /* pairs per slot (1..2^30; 2^22) */
} cc_server_opt;
void cc_server_default_opt(cc_server_opt *opt);
cc_status cc_server_create(cc_incr *h, const cc_server_opt *opt, cc_server **out);
cc_status cc_server_submit(cc_server *s, const uint32_t *inserts, uint64_t k, const uint32_t *queries, uint64_t q,
                           uint8_t *answers, uint64_t *ticket_out);
cc_status cc_server_wait(cc_server *s, uint64_t ticket, double *latency_ms_out);
cc_status cc_server_destroy(cc_server *s);

/* Learned variant selector (no counterpart in the paper, whose Section 4.7
 * offers a hand-made decision tree): an FP32 MLP 16 -> 64 -> 64 -> 12 with
 * ReLU, trained on the GPU by these kernels.  It only picks which
 * combination to run; labels never depend on it.
 * Parameter block (DEVICE float[CC_MLP_NPARAM]): mu[16], sigma[16] (input
 * standardisation), W1[16][64], b1[64], W2[64][64], b2[64], W3[64][12],
 * b3[12]; W[i][j] maps input i to output j.  X: DEVICE float[B][16].
 * cc_mlp_init: Glorot-uniform weights from counter-based draws of `seed`,
 *   zero biases, mu = 0, sigma = 1.
 * cc_mlp_set_norm: mu, sigma <- mean, standard deviation of X's columns.
 * cc_mlp_forward: logits float[B][12]; acts (may be NULL) float[B][128]
 *   gets both hidden layers for cc_mlp_backward.
 * cc_mlp_soft_targets: targets[B][12] from measured times[B][12]:
 *   q_c proportional to exp(-(t_c / min_c t_c - 1) / tau).
 * cc_mlp_backward: grads float[CC_MLP_NPARAM] <- gradient of the mean
 *   cross-entropy between softmax(logits) and the targets (zero for mu,
 *   sigma); *loss (DEVICE float, may be NULL) <- that mean.  Per-sample
 *   gradients are summed in a fixed order (deterministic).
 * cc_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the
 *   trained parameters; m, v: DEVICE float[CC_MLP_NPARAM], zero at step 1.
 * cc_mlp_predict: class_out DEVICE int32[B] <- argmax of the logits. */
#define CC_MLP_IN 16
#define CC_MLP_HID 64
#define CC_MLP_OUT 12
#define CC_MLP_NPARAM (2 * CC_MLP_IN + CC_MLP_IN * CC_MLP_HID + CC_MLP_HID + CC_MLP_HID * CC_MLP_HID + \
                       CC_MLP_HID + CC_MLP_HID * CC_MLP_OUT + CC_MLP_OUT)
/* Selector features of a graph (same conventions as cc_static; n >= 1):
 * feat_out (DEVICE float[16]) <- the features the selected path
 * (cc_select_static) computes on its way, from the k-out (k = 2, `seed`)
 * sample it starts with: 0 log2(n+1), 1 log2(m+1), 2 m/n, 3 log2(max
 * degree + 1), 4 degree variance / mean^2, 5-7 fractions of vertices of
 * degree 0, 1, 2, 8 fraction of degree 3..16, 9 fraction of degree > 64,
 * 10 share of edges at vertices of degree > 64, 11 size of the frequent
 * sampled cluster L_max / n, 12 vertices outside their own singleton after
 * sampling / n, 13 edges left for the finish (edges out of vertices not in
 * L_max) / m, 14 light candidates of the finish (not in L_max, degree
 * 1..32) / n, 15 parent steps walked per non-root by the sampling's last
 * compression (how deep the sampled trees were).  Stream-ordered. */
cc_status cc_features(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                      uint64_t seed, float *feat_out, void *stream);
/* The selected static path (the learned selector; no counterpart in the
 * paper, whose Section 4.7 picks by a hand-made decision tree).  Labels
 * exactly as cc_static, by one of 12 classes c = 4 * sampling + finish:
 * sampling 0 k-out (k = 2), 1 BFS (3 tries), 2 LDD (beta 0.2); finish 0
 * UF-Rem-CAS (FindNaive, SplitAtomicOne), 1 UF-Async (FindSplit), 2 SV,
 * 3 Liu-Tarjan PRF.  The default class 0's k-out sample is computed first;
 * the features (cc_features) come from it and the MLP `params` (DEVICE
 * float[CC_MLP_NPARAM]) picks the class on the device.  The host waits
 * for the choice only (not for the labels): class 0 and the other k-out
 * classes continue on the same sample and candidate lists; BFS and LDD
 * classes run the static path from scratch.  force_class in [0, 12)
 * overrides the MLP (params may then be NULL); -1 uses it.  feat_out
 * (DEVICE float[16], may be NULL) receives the features; *class_out (host,
 * may be NULL) the class run.  The labels are stream-ordered on `stream`. */
cc_status cc_select_static(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                           const float *params, int force_class, uint64_t seed, uint32_t *labels_out,
                           float *feat_out, int32_t *class_out, void *stream);
cc_status cc_mlp_init(float *params, uint64_t seed, void *stream);
cc_status cc_mlp_set_norm(float *params, const float *X, uint32_t B, void *stream);
cc_status cc_mlp_forward(const float *params, const float *X, uint32_t B, float *logits, float *acts, void *stream);
cc_status cc_mlp_soft_targets(const float *times, uint32_t B, float tau, float *targets, void *stream);
cc_status cc_mlp_backward(const float *params, const float *X, const float *acts, const float *logits,
                          const float *targets, uint32_t B, float *grads, float *loss, void *stream);
cc_status cc_mlp_adam(float *params, const float *grads, float *m, float *v, uint32_t step, float lr, void *stream);
cc_status cc_mlp_predict(const float *params, const float *X, uint32_t B, int32_t *class_out, void *stream);

/* Self-check of the bounded grid barrier (the wait the persistent BFS
 * levels use): a cooperative launch of one block per SM meets at the
 * barrier three times.  skip_block >= 0 names a block that leaves without
 * arriving; the others then give up after wait_ms (1..4000), flag
 * CC_DEVERR_NONCONVERGED and leave, and the call returns
 * CC_ERR_NONCONVERGED with *blocks_passed_out = 0 (host) and a usable
 * context.  skip_block < 0: every block passes, CC_OK.  Synchronises. */
cc_status cc_selftest_grid_barrier(int skip_block, uint32_t wait_ms, uint32_t *blocks_passed_out, void *stream);

/* Synchronise `stream`, then read and clear the per-device sticky error
 * word (CC_DEVERR_* bits) into *bits_out (host; may be NULL).  Returns
 * CC_OK when the word was 0, else the matching status. */
cc_status cc_device_error(void *stream, uint32_t *bits_out);

/* Test hook: cap on the iterations of one device loop (a find, a union, a
 * round loop).  0 restores the default (2n + 1024 steps, 4096 rounds). */
void cc_set_iteration_cap(uint64_t cap);

/* Instrumentation (the library's own tracing; no paper counterpart beyond
 * its per-phase timings).  Every kernel launch increments a process-wide
 * counter (cc_launch_count).  While profiling is enabled, each launch is
 * also bracketed by CUDA events on its stream; cc_profile_read waits for
 * those events and returns per-kernel totals (name, launches, milliseconds)
 * accumulated since profiling was enabled, up to `max` entries, returning
 * the number of kernels.  Enabling resets the totals. */
typedef struct cc_kernel_time {
    char name[48];
    uint64_t launches;
    double ms;
} cc_kernel_time;
void cc_profile_enable(int on);
int cc_profile_read(cc_kernel_time *out, int max);
uint64_t cc_launch_count(void);

const char *cc_status_str(cc_status s);
const char *cc_version(void);
/* The compute capability of the device code the runtime loaded for this
 * library on the current device, as major * 10 + minor (103 for the
 * sm_103a build); no paper counterpart.  Needs a device: CC_ERR_CUDA
 * without one. */
cc_status cc_binary_version(int *version_out);

#ifdef __cplusplus
}
#endif
#endif /* CONNECTIT_GB_H */
