/*
 * cubics.h — C ABI of the GB300 CUBICS hot path (arxiv 1909.09213).
 *
 * A problem is the CSP triple (X, D, C) of Section 1.1: `csp_create` makes the variables X
 * with their domains D, `csp_remove_value` cuts arbitrary holes in D, and the `csp_post_*`
 * calls add the constraints C.  The host builds and encodes the problem and moves it to the
 * GPU once; labeling, propagation and backtracking then run entirely on the device, and
 * only solutions and statistics come back (Section 2.1).
 *
 * Conventions shared by every call:
 *   - every function returns an int status (CSP_OK or a negative CSP_E* code); on error the
 *     handle is unchanged;
 *   - pointers named `host` point to host memory, `dev` to device memory; the library copies
 *     host arrays it is given and never keeps or frees caller pointers;
 *   - the library never allocates device memory: the caller binds a device workspace of
 *     `csp_workspace_bytes` bytes (e.g. a torch.uint8 CUDA tensor) and a CUDA stream;
 *   - handles are not thread-safe; there is no CPU fallback: without a usable GPU every
 *     device call returns CSP_ECUDA.
 *
 * Domains on the device are bitsets: all variables of one problem share the window
 * lo0 .. lo0 + 32*W - 1 (lo0 = min lo_i, W = ceil(span/32) words, span <= 256), and bit k of a
 * domain stands for the value lo0 + k.  `csp_layout` reports n, W and lo0.
 */
#ifndef CUBICS_H
#define CUBICS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CSP_OK = 0,
    CSP_EINVAL = -1,    /* bad argument: variable index, empty domain, x == y table, ... */
    CSP_ENOMEM = -2,    /* bound workspace smaller than csp_workspace_bytes */
    CSP_ETOOBIG = -3,   /* beyond the supported sizes (n > 1024, span > 256, overflow risk) */
    CSP_ECUDA = -4,     /* CUDA error or no device */
    CSP_ELIMIT = -5,    /* node or time limit reached; statistics are partial */
    CSP_ETIMEOUT = -6,  /* a device-side wait for work exceeded wait_limit_ns */
    CSP_ESTATE = -7     /* call out of order (e.g. solve before bind) */
};

enum { CSP_ALL = 0, CSP_FIRST = 1, CSP_PROPAGATE = 2 };
enum { CSP_BR_FIRST_FAIL = 0, CSP_BR_LEARNED = 1 };

/* test hook flags for csp_limits.flags */
enum { CSP_F_NO_DONATE = 1 };   /* workers never share subtrees (exercises the wait limit) */

typedef struct csp csp_t;
typedef struct csp_batch csp_batch_t;

typedef struct {
    int64_t node_limit;      /* stop after about this many nodes (batches: per instance, which
                                then reports CSP_ELIMIT); 0 = none */
    int64_t time_limit_ns;   /* stop after this device time; 0 = none */
    int64_t wait_limit_ns;   /* bound on every device-side wait; 0 = 60 s */
    int32_t flags;           /* CSP_F_* */
    int32_t reserved;
} csp_limits;

/* Launch shape of the search kernel.  0 fields are chosen by the library. */
typedef struct {
    int32_t blocks;           /* persistent blocks; 0 = resident blocks on every SM */
    int32_t warps_per_block;  /* workers per block (one warp each); 0 = 8.  A block must fit
                                 the search kernel's register budget (the first-fail kernels
                                 admit 25 warps for one-word domains and 21 for wider ones;
                                 the one for one-word int_ne problems of at most 32
                                 variables admits 32): larger blocks make planning fail
                                 with CSP_EINVAL */
    int32_t smem_levels;      /* search-stack levels kept in shared memory per worker */
    int32_t queue_records;    /* capacity of each work queue (power of two) */
    int32_t threads_per_node; /* 16: two sibling nodes per warp, a half-warp each: search
                                 of all solutions of a one-word int_ne problem of at most 16
                                 variables (the register-held kernel, first-fail brancher);
                                 anything else with 16 is CSP_EINVAL.  The two siblings'
                                 fixpoints share every instruction; the search visits the
                                 same nodes (same counts and hashes), child 0's subtree
                                 first, and max_depth counts stack levels (up to 2n - 1).
                                 32: a warp per node.  0: the library's choice (16 where it
                                 applies, else 32).  64..1024 (a multiple of 32):
                                 csp_propagate gives each domain state a whole block, its
                                 warps sharing out the constraints of each kind
                                 (constraint-parallel propagation of one node too large for
                                 a warp, Section 2.2's grouping by kind); a search plan with
                                 it is CSP_EINVAL */
    int32_t split_depth;      /* all-solution search of one problem (csp_solve / csp_launch):
                                 k = 1..8: the first k levels are expanded on the device (one
                                 fixpoint and one expansion kernel per level; csp_launch then
                                 waits for the device between levels) and the subtrees below
                                 them are solved like a batch, each block's warps sharing one
                                 subtree through the block's own queue; 0 = the library's
                                 choice (3); -1 = all workers share one queue of the whole
                                 tree.  Same counts and hashes either way; no effect on
                                 first-solution search, partitions, the learned brancher
                                 (CSP_BR_LEARNED) or csp_solve_noalloc */
    int32_t domain_words;     /* search bitset width: 0 = the problem's own (csp_layout's W);
                                 1, 2, 4 or 8 words per domain, at least the problem's own:
                                 the search runs with wider domains (the same values, upper
                                 words empty), the autotuner's width axis.  The register-held
                                 kernel and two nodes per warp need one-word domains, so
                                 threads_per_node = 16 with a wider width is CSP_EINVAL.
                                 csp_propagate, csp_root_domains and csp_layout keep the
                                 problem's own width.  A batch runs at the widest width of its
                                 problems: any other nonzero value is CSP_EINVAL there */
} csp_tiling;

typedef struct {
    uint64_t nodes;          /* fixpoint calls, root included */
    uint64_t fails;          /* fixpoint calls that emptied a domain */
    uint64_t solutions;      /* all solutions (CSP_ALL) or 1/0 (CSP_FIRST) */
    uint64_t sol_hash_sum;   /* sum over solutions of the solution hash (mod 2^64) */
    uint64_t sol_hash_xor;   /* xor over solutions of the solution hash */
    uint64_t prop_evals;     /* propagator evaluations */
    uint64_t steals;         /* subtrees handed from one worker to another */
    uint64_t spills;         /* search-stack levels moved from shared to global memory */
    int32_t max_depth;       /* deepest open search level seen */
    int32_t status;          /* last call's status */
    double ms;               /* device time of the last search launch */
    int64_t stored;          /* solutions written to sol_out */
    int32_t workers;         /* workers (warps) of the last launch */
    int32_t blocks;          /* blocks of the last launch */
    int64_t h2d_bytes;       /* host-to-device bytes of the last upload (batches: uploaded
                                since the previous successful collect) */
    int64_t d2h_bytes;       /* device-to-host bytes of the last collect */
    uint64_t wait_ns;        /* summed over workers: time spent waiting for work */
    uint64_t rounds;         /* fixpoint rounds (propagation passes over the changed scopes) */
    double kernel_ms;        /* device time of the search kernel alone (ms also covers the
                                level expansion of a split search) */
    int64_t units;           /* subtrees the last search solved: those below the expanded
                                levels of a split search, else 1; a batch: its problems;
                                0 after csp_propagate */
} csp_stats_t;

typedef struct {
    int32_t status;          /* 1 SAT, 0 UNSAT, < 0 error (CSP_ELIMIT, ...) */
    int32_t n;               /* number of variables */
    uint64_t nodes;          /* nodes spent on this instance */
    uint64_t fails;
    uint64_t solutions;      /* CSP_ALL: every solution; CSP_FIRST: 1 when SAT */
    int64_t sol_offset;      /* first solution of the instance: values at sol + sol_offset */
    double ms;               /* device time from the start of the instance's search (its block
                                took it) to its verdict */
} csp_result;

/* ---------------------------------------------------------------- model (host only) */

/* Create X = {x_0..x_{n-1}} with D_i = {lo[i]..hi[i]} (Section 1.1).  Every hi[i] - lo[i]
 * must be in 0..255 and all values must fit one window of 256 consecutive integers.
 * lo, hi: host arrays of n_vars entries.  Returns CSP_EINVAL for n_vars < 1 or hi < lo,
 * CSP_ETOOBIG for n_vars > 1024 or a window wider than 256. */
int csp_create(csp_t **out, int32_t n_vars, const int32_t *lo, const int32_t *hi);

/* Remove `value` from D_var (arbitrary finite domains, Section 1.1).  Values outside the
 * domain are ignored.  CSP_EINVAL for a bad index. */
int csp_remove_value(csp_t *h, int32_t var, int32_t value);

/* x != y + c; y < 0 posts the unary x != c.  Propagation: when one side is fixed, the value
 * it forbids is removed from the other (Section 1.1, constraint propagation). */
int csp_post_int_ne(csp_t *h, int32_t x, int32_t y, int32_t c);

/* sum_{t<k} coef[t] * x_{vars[t]} <= rhs, bounds-consistent.  Repeated variables are merged
 * and zero coefficients dropped.  coef, vars: host arrays of k entries.  CSP_ETOOBIG when
 * sum |coef| * max |value| + |rhs| could exceed 2^30. */
int csp_post_int_lin_le(csp_t *h, int32_t k, const int32_t *coef, const int32_t *vars,
                        int32_t rhs);

/* all different over k distinct variables: fixed values are removed from the other
 * members; fails when two members share a fixed value or when fewer than k values remain
 * in the union of their domains.  vars: host array of k entries; repeats are CSP_EINVAL. */
int csp_post_alldiff(csp_t *h, int32_t k, const int32_t *vars);

/* all different over k <= 32 distinct variables, bounds-consistent (Section 4, second
 * direction: a costlier propagation that prunes more): a bound of a member's domain stays only
 * when the other members can take distinct values within their own [min, max] while the
 * member takes that bound; holes are kept, so a bound that goes moves to the next value of
 * the domain.  Complements csp_post_alldiff (value elimination); post both for both.
 * vars: host array of k entries; repeats are CSP_EINVAL, k > 32 is CSP_ETOOBIG. */
int csp_post_alldiff_bc(csp_t *h, int32_t k, const int32_t *vars);

/* Binary relation as a tuple set (c2 of Section 1.1), arc-consistent.  allowed: host array
 * of (hi_x - lo_x + 1) rows of row_words uint32 words; bit b of row a allows the pair
 * (lo_x + a, lo_y + b).  row_words >= ceil((hi_y - lo_y + 1) / 32).  x == y is CSP_EINVAL. */
int csp_post_table(csp_t *h, int32_t x, int32_t y, const uint32_t *allowed, int32_t row_words);

/* Device domain layout: n variables, W uint32 words per domain, bit k = value lo0 + k. */
int csp_layout(const csp_t *h, int32_t *n, int32_t *W, int32_t *lo0);

/* Root domains as the kernels receive them: `host_out` gets n * W words in the layout of
 * csp_layout.  Host only (no device needed).  CSP_EINVAL for NULL arguments. */
int csp_root_domains(const csp_t *h, uint32_t *host_out);

/* A new handle holding a copy of the model of `src` (variables, domains, constraints,
 * tiling, brancher and its weights, partition); it is unbound and independent of `src`.
 * The paper has no counterpart: large neighbourhood search (Section 4, first direction)
 * builds each neighbourhood as a copy of the problem with some domains reset.  Host only. */
int csp_clone(const csp_t *src, csp_t **out);

/* Restrict D_{vars[t]} to {values[t]} for t < count (the domain becomes empty when the value
 * is not in it).  vars, values: host arrays of count entries.  CSP_EINVAL for a bad index
 * (nothing is changed then).  Host only. */
int csp_fix_values(csp_t *h, int32_t count, const int32_t *vars, const int32_t *values);

/* ---------------------------------------------------------------- device (single problem) */

/* Launch shape; NULL or zero fields restore the library's choice.  Changes the workspace
 * size. */
int csp_set_tiling(csp_t *h, const csp_tiling *t);

/* Bytes of device workspace needed for `mode` (CSP_ALL / CSP_FIRST with up to `cap` stored
 * solutions, or CSP_PROPAGATE with cap = number of domain states) under the current tiling. */
int csp_workspace_bytes(const csp_t *h, int32_t mode, int64_t cap, size_t *bytes);

/* Bind a device workspace (dev, >= csp_workspace_bytes, 256-byte aligned) and a CUDA stream
 * (cudaStream_t as void*, NULL = legacy default stream).  The caller owns both and must keep
 * them alive until the handle is destroyed or rebound. */
int csp_bind(csp_t *h, void *dev, size_t bytes, void *cuda_stream);

/* Share one search tree between nparts ranks (search-space partitioning, Section 1.3): the
 * root is propagated by every rank, and its children (the values of the root's branching
 * variable, ascending) are dealt round-robin, rank `part` exploring positions
 * part, part + nparts, ...  The root's own node, fail or solution is counted by part 0 only,
 * so summing the ranks' counts and hash sums (and xoring their hash xors) gives the
 * undivided search's results.  Default 0 of 1.  CSP_EINVAL unless 0 <= part < nparts. */
int csp_set_partition(csp_t *h, int32_t part, int32_t nparts);

/* Branching heuristic: CSP_BR_FIRST_FAIL (smallest domain, lowest index) or
 * CSP_BR_LEARNED with the brancher's bf16 weights (host array, csp_brancher_params()
 * values; NULL keeps the loaded weights).  Learned ordering changes only exploration order. */
int csp_set_brancher(csp_t *h, int32_t kind, const uint16_t *bf16_weights);

/* Search (Sections 1.1 and 2.1): d-way branching on the chosen variable, values ascending,
 * every node propagated to its fixpoint on the GPU, backtracking on device.  CSP_ALL counts
 * every solution and stores up to cap of them (any `cap` of them, unordered); CSP_FIRST stops
 * at the first.  sol_out: host array of cap * n int32 values (may be NULL when cap == 0).
 * Encodes and uploads the problem, launches, waits, and copies results back.  lim may be NULL. */
int csp_solve(csp_t *h, int32_t mode, int64_t cap, int32_t *sol_out, const csp_limits *lim);

/* The device part of csp_solve alone: requires a previous csp_solve or csp_upload with the
 * same mode and cap; enqueues the search on the bound stream and returns without waiting.
 * Results stay in the workspace until csp_collect. */
int csp_upload(csp_t *h, int32_t mode, int64_t cap);
int csp_launch(csp_t *h, const csp_limits *lim);
int csp_collect(csp_t *h, int32_t *sol_out);

/* One fixpoint per domain state (test hook, and the level expansion of a depth-k search-space
 * partition; Section 1.1, constraint propagation).  dom_in, dom_out: host arrays of
 * count * n * W words (layout of csp_layout); failed: host array of count int32 (1 = some
 * domain became empty; dom_out is then unspecified).  A warp per state, or a block per state
 * when csp_tiling.threads_per_node > 32.  csp_stats afterwards: nodes = count, fails = the
 * failed states, ms = the kernel's device time. */
int csp_propagate(csp_t *h, int32_t count, const uint32_t *dom_in, uint32_t *dom_out,
                  int32_t *failed);

int csp_stats(const csp_t *h, csp_stats_t *out);
void csp_destroy(csp_t *h);
const char *csp_strerror(int code);

/* ---------------------------------------------------------------- batches */

/* Many problems solved by one persistent launch: each block takes the next instance from an
 * atomic ticket and its warps share that instance's subtrees.  The handles must outlive the
 * batch; their models are encoded at csp_batch_create. */
int csp_batch_create(csp_batch_t **out, csp_t *const *hs, int32_t count);

/* A batch of `count` copies of `base` that differ only in their root domains: copy i starts
 * from host_roots[i*n*W .. (i+1)*n*W) intersected with the root domains of `base` (layout of
 * csp_layout).  The model is encoded once and the copies share its constraints.  `base` must
 * outlive the batch and stay unchanged.  The paper has no counterpart: the neighbourhoods of
 * large neighbourhood search (Section 4) are such copies.  Host only. */
int csp_batch_create_roots(csp_batch_t **out, csp_t *base, int32_t count,
                           const uint32_t *host_roots);
int csp_batch_set_tiling(csp_batch_t *b, const csp_tiling *t);
int csp_batch_workspace_bytes(const csp_batch_t *b, int32_t mode, size_t *bytes);
int csp_batch_bind(csp_batch_t *b, void *dev, size_t bytes, void *cuda_stream);
/* out: host array of count results; sol: host array of csp_batch_solution_words() int32
 * (first solution per SAT instance), may be NULL.  use_graph != 0 replays a CUDA graph. */
int csp_batch_solve(csp_batch_t *b, int32_t mode, const csp_limits *lim, int32_t use_graph,
                    csp_result *out, int32_t *sol);
int csp_batch_launch(csp_batch_t *b, const csp_limits *lim, int32_t use_graph);
int csp_batch_collect(csp_batch_t *b, csp_result *out, int32_t *sol);
int64_t csp_batch_solution_words(const csp_batch_t *b);
/* Brancher of every instance of the batch (as csp_set_brancher). */
int csp_batch_set_brancher(csp_batch_t *b, int32_t kind, const uint16_t *bf16_weights);
/* Subtree logging for training the learned brancher (no counterpart in the paper): while
 * searching, every completed search level whose hash (worker, node count) is 0 mod `sample`
 * appends 17 floats to log_dev — the 16 features of the level's branching variable when it
 * was chosen, then log2 of the number of nodes in the level's subtree — at the index returned
 * by an atomic increment of *count_dev (caller zeroes it), up to cap entries.  Logging keeps
 * every subtree with the worker that opened it (no donation, no helping blocks), so use one
 * warp per block.  cap = 0 turns logging off.  log_dev, count_dev: device pointers. */
int csp_batch_set_log(csp_batch_t *b, float *log_dev, unsigned long long *count_dev, int64_t cap,
                      uint32_t sample);
int csp_batch_stats(const csp_batch_t *b, csp_stats_t *out);
void csp_batch_destroy(csp_batch_t *b);

/* ---------------------------------------------------------------- learned brancher network */

/* The network that scores branching variables: 16 features -> 64 -> 64 -> 1, ReLU, bfloat16
 * weights and activations, fp32 accumulation (no counterpart in the paper; it only reorders
 * the search).  Flat parameters (CSP_MLP_PARAMS values): W1 [16][64] row-major, b1[64],
 * W2 [64][64], b2[64], w3[64], b3[1].  All pointers below are device pointers; every call is
 * asynchronous on cuda_stream. */
#define CSP_MLP_PARAMS 5313
#define CSP_MLP_PACKED_WORDS 2948

/* Fragment-ordered copy of the bf16 parameters (packed_dev: CSP_MLP_PACKED_WORDS uint32). */
int csp_mlp_pack(const uint16_t *params_dev, uint32_t *packed_dev, void *cuda_stream);
/* scores_dev[r] for the rows x16 features of X_dev (fp32, rounded to bf16 on load), computed
 * with warp-level tensor-core tiles of 16 rows. */
int csp_mlp_forward(const uint32_t *packed_dev, const float *X_dev, int32_t rows, float *scores_dev,
                    void *cuda_stream);
/* Mean squared error of the scores against y and its gradient (grad_dev: CSP_MLP_PARAMS fp32;
 * loss_dev: 1 fp32 or NULL) for fp32 master weights that are rounded to bf16 as in inference. */
int csp_mlp_grad(const float *master_dev, const float *X_dev, const float *y_dev, int32_t rows,
                 float *grad_dev, float *loss_dev, void *cuda_stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8; step counts from 1) on master_dev with moments
 * m_dev, v_dev; params_dev (may be NULL) receives the new bf16 weights. */
int csp_mlp_adam(float *master_dev, float *m_dev, float *v_dev, const float *grad_dev, int32_t step,
                 float lr, uint16_t *params_dev, void *cuda_stream);

/* ---------------------------------------------------------------- allocation-free search */

/* csp_solve for callers that cannot allocate device memory.  Some callers may not call
 * cudaMalloc at all: a plug-in loaded into a host application that owns every device
 * allocation (through its own pool, under its own memory cap), or a latency-bound loop in
 * which an allocation may block or synchronise the device.  The paper has no counterpart;
 * this is a library convenience.
 *
 * Instead of a bound workspace, the search uses a scratch array inside the library's own
 * device image (CSP_NOALLOC_SCRATCH_BYTES = 16 MiB, reserved on every GPU that loads the
 * library until the process exits).  The call performs no cudaMalloc, cudaFree,
 * cudaMallocHost or other device/pinned allocation: the encoded problem is copied from
 * ordinary host memory straight into the array, and results are copied back the same way.
 * Inputs and outputs are the caller's: the handle h (model built with csp_create/post),
 * sol_out (host, cap * n int32; may be NULL when cap == 0) and the statistics read back
 * with csp_stats (stats.ms is 0: no events are created).  cuda_stream: cudaStream_t as
 * void* (NULL = legacy stream); the call waits for the search on it before returning.
 * The handle's own binding and upload (csp_bind, csp_upload) are neither used nor
 * changed, whatever the call returns.
 *
 * The first call on each device does a one-time set-up: it looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  Every call on a device shares the one array and leaves its contents
 * behind; the counters that must start at zero are cleared by each call.  Calls that
 * overlap on the GPU (other host threads, other streams) race on the array: serialise them.
 * The call waits for the device and copies from pageable host memory, which a stream
 * capture does not allow: on a capturing stream it returns CSP_ESTATE at once, doing nothing
 * (the capture stays valid).
 * Returns CSP_ENOMEM when the problem, the launch shape (csp_set_tiling) and cap need more
 * than the array holds, plus the error codes of csp_solve. */
#define CSP_NOALLOC_SCRATCH_BYTES (16u << 20)
int csp_solve_noalloc(csp_t *h, int32_t mode, int64_t cap, int32_t *sol_out,
                      const csp_limits *lim, void *cuda_stream);

/* ---------------------------------------------------------------- measurement */

/* Shared-memory bandwidth of the current device (a measurement helper with no counterpart
 * in the paper; it is the denominator of the search kernel's roofline).  Every SM streams
 * 128-bit ld.shared over a 64 KB buffer; *gbs receives bytes read / kernel time in GB/s
 * (best of `reps` launches).  dev_out: device buffer of at least 16 bytes that receives a
 * checksum so the loads are not optimised away.  Synchronises `cuda_stream`. */
int csp_probe_smem_bandwidth(void *dev_out, void *cuda_stream, int32_t reps, double *gbs);

#ifdef __cplusplus
}
#endif
#endif /* CUBICS_H */
