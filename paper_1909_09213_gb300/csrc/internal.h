// Internal layout shared by the library's host encoder and its CUDA kernels.
//
// One problem is encoded as a flat array of uint32 words ("instance block").  The first
// HDR_WORDS words are a header of offsets (in words, from the start of the block); then the
// constraint data, which blocks stage into shared memory; then the root domains.
//
// Domains are bitsets of W words: bit k of variable i's domain (word i*W + k/32) stands for
// the value lo0 + k.  All variables of an instance share lo0 and W.
#pragma once
#include <stdint.h>

namespace cubics {

constexpr int MAX_VARS = 1024;          // NW = ceil(n/32) <= 32 event words per worker
constexpr int MAX_W = 8;                // 256-value window
constexpr int HDR_WORDS = 48;
constexpr int ADB_MAX = 32;             // members of a bounds-consistent alldifferent group
constexpr uint32_t FLAG_TRIVIAL_FAIL = 1u;  // a row with no terms and rhs < 0
constexpr uint32_t FLAG_NE_ONLY = 2u;       // int_ne constraints only (no lin, alldiff, table)
constexpr uint32_t FLAG_NE_REG = 4u;        // also one word per domain and n <= 32: the search
                                            // can hold a node's domains in registers, one
                                            // variable per lane (offset masks at H_OFF_NEMASK)
constexpr int WS_WORDS = 92;            // per-warp shared bookkeeping (events, counters)
// Deferred solution hashing of the register kernel: up to HB_SOLS solutions of at most 32
// one-byte values (offsets from lo0), HB_STRIDE words apart (8 words of values and one of
// padding, so that neither the byte writes of one solution nor the lanes' reads of one word
// each of different solutions meet in a bank)
constexpr int HB_SOLS = 32;
constexpr int HB_STRIDE = 9;
constexpr int HB_WORDS = HB_SOLS * HB_STRIDE;
// search kernel kinds
constexpr int KERN_PLAIN = 0;           // first-fail, domains in shared memory
constexpr int KERN_EXT = 1;             // learned brancher and/or subtree logging
constexpr int KERN_REG = 2;             // FLAG_NE_REG problems, domains in registers

enum Hdr {
    H_N = 0, H_W, H_LO0, H_S, H_NW, H_FLAGS,
    H_N_UN, H_OFF_UN,                 // unary x != c: (x | bit << 16)
    H_OFF_ADJ_START, H_OFF_ADJ,       // ne adjacency: n+1 starts; (other | (uint16)off << 16)
    H_N_LIN, H_OFF_LIN_ROW, H_OFF_LIN_TERM, H_LIN_MW, H_OFF_LIN_MASK,
    H_N_AD, H_OFF_AD_ROW, H_OFF_AD_MEM, H_AD_MW, H_OFF_AD_MASK,
    H_N_TAB, H_OFF_TAB,
    H_OFF_ROOT, H_CONS_WORDS, H_TOTAL, H_R, H_N_NE,
    H_OFF_VFEAT,                      // per variable VFEAT_WORDS words of static feature data
    H_OFF_NB_START, H_OFF_NB,         // neighbour lists: n+1 starts; neighbour indices
    H_MAXDEG,                         // largest constraint degree of a variable
    H_OFF_NEMASK,                     // FLAG_NE_REG: n x 32 offset masks of 2 words (below)
    H_N_ADB, H_OFF_ADB_ROW, H_OFF_ADB_MEM, H_ADB_MW, H_OFF_ADB_MASK,   // bounds-consistent
                                      // alldifferent groups, laid out as the alldiff ones
    H_COUNT
};

// static feature data of a variable: offset of its own lo from lo0, initial domain size,
// constraint degree, counts of ne / lin / alldiff / table constraints, mean forbidden
// fraction of its tables (float bits)
constexpr int VFEAT_WORDS = 8;
constexpr int N_FEATURES = 16;
static_assert(H_COUNT <= HDR_WORDS, "header too long");

// int_ne offset masks (FLAG_NE_REG): for a fixed variable v and a variable i, the 64-bit
// mask at words H_OFF_NEMASK + 2 (32 v + i) (low word first) has bit off + 31 set when some
// int_ne makes "x_v fixed to bit a" remove bit a + off from D(x_i) (|off| <= 31; larger
// offsets never meet a one-word domain).  Indexed fixed variable first, so that the 32 lanes
// of a warp read the masks of one fixed variable from consecutive words.
// lin row: 3 words (first term, number of terms, rhs); term: 2 words (coef, var)
// alldiff group (both kinds): 2 words (first member, number of members)
// table: 4 words (x, y, word offset of R, word offset of C); R and C hold 32*W rows of W
//        words: R row a = values of y compatible with x = lo0 + a, C row b the transpose.

// Search-stack level / work record: R words = S domain words, W words of values still to
// try, one word with the branching variable (-1: the record is a node to propagate), and
// `extra` words (subtree logging: the node count at the level's creation and the chosen
// variable's 16 features).
__host__ __device__ inline int record_words(int S, int W, int extra = 0) {
    return (S + W + 1 + extra + 3) & ~3;
}
constexpr int LOG_EXTRA = 1 + 16;

struct Team {                 // one work-sharing group (whole grid or one block)
    int32_t work;             // records queued or being explored
    int32_t found;            // 1: CSP_FIRST solution recorded; 2: the instance hit its node limit
    int32_t inst;             // instance index (batch mode)
    int32_t helpers;          // batch mode: blocks of other teams that joined (or are joining)
    unsigned long long progress;  // batch mode: nodes spent on the instance (limit accounting)
    int32_t pad1[26];
    uint32_t head;            // consumer tickets (own 128-byte line)
    int32_t pad2[31];
    uint32_t tail;            // producer positions (own 128-byte line)
    int32_t pad3[31];
    uint32_t promised;        // records pushed or promised by donors (own line); head -
                              // promised > 0: workers wait for records nobody has promised
    int32_t pad4[31];
    // subtrees taken from the queue, by the share of unfixed variables in the record (bin
    // u * UBINS / (n + 1)): how many, and their nodes in total
    uint32_t ucnt[32];
    unsigned long long usum[32];
    unsigned long long xns, xnodes;   // time and nodes spent in finished records
    int32_t pad5[28];
};
constexpr int UBINS = 32;
static_assert(sizeof(Team) == 1024, "Team is eight 128-byte lines");

struct GState {               // counters of one launch
    unsigned long long nodes, fails, solutions, hsum, hxor, evals, steals, spills;
    unsigned long long stored;        // solution slots taken
    unsigned long long node_progress; // for the node limit
    unsigned long long wait_ns;       // summed over workers: time spent waiting for work
    unsigned long long rounds;        // fixpoint rounds
    int32_t max_depth;
    int32_t status;                   // 0 ok, else CSP_E*
    int32_t abort;                    // global stop
    int32_t ticket;                   // next batch instance
    int32_t pad[20];
};

struct InstResult {
    int32_t status;           // 1 SAT, 0 UNSAT, < 0 error
    int32_t n;
    unsigned long long nodes, fails, solutions;
    int64_t sol_offset;
    long long t_start, t_end; // global timer (ns) when the owning block started the instance and
                              // when its verdict became final
};

struct SearchArgs {
    const uint32_t *arena;    // instance blocks
    const int64_t *inst_off;  // word offset of each instance block
    const int64_t *sol_off;   // batch: offset of each instance's solution slot in `sols`
    int32_t n_inst;
    int32_t mode;             // 0 all, 1 first
    int32_t batch;            // 0: one team = grid; 1: one team per block, instance tickets
    int32_t lsm;              // stack levels in shared memory per worker
    int32_t rmax;             // record words (max over instances)
    int32_t depth;            // stack levels per worker (max n + 1)
    int32_t stage_words;      // shared-memory words reserved for constraint data
    int32_t qmask;            // queue capacity - 1
    int32_t flags;
    int32_t warps;            // workers per block
    int32_t part, nparts;     // single mode: explore only the root children of rank part
    GState *g;
    Team *teams;
    uint32_t *qseq;           // per team: qcap sequence words
    uint32_t *qrec;           // per team: qcap records of rmax words
    uint32_t *spill;          // per worker: depth records of rmax words
    int32_t *sols;
    int64_t cap;
    InstResult *results;
    long long node_limit;
    long long deadline_ns;    // time limit from each worker's start, 0 = none
    long long wait_limit_ns;
    const uint32_t *mlp;      // learned brancher: packed network weights, NULL = first-fail
    int32_t mlp_off;          // SM word offset of the staged weights, -1 = first-fail
    int32_t feat_words;       // per-warp words of the learned brancher's feature tile
    int32_t warp_base;        // SM word offset of warp 0's area
    int32_t list_words;       // per-warp words of the scheduled-table list (one-word tables)
    int32_t log_extra;        // subtree logging: LOG_EXTRA extra record words, else 0
    uint32_t log_sample;      // log one completed level in log_sample (hash of worker, count)
    float *logbuf;            // log entries of 17 floats: 16 features, log2 subtree nodes
    unsigned long long *log_count;
    long long log_cap;
    const uint32_t *roots;    // batch: root domains of instance i at roots + i * S (all
                              // instances sharing one block); NULL: each block's own roots
    int32_t global_limits;    // batch: the node limit counts all instances together and stops
                              // the launch (the instances are parts of one search)
    int32_t hash_words;       // per-warp words of the deferred solution-hash buffer (register
                              // kernel: HB_SOLS solutions of HB_STRIDE words), else 0
    int32_t pairs;            // register kernel, all solutions, n <= 16: two sibling nodes per
                              // warp (the stack has room for 2n levels)
    int32_t pad_args;
};

// One level of the depth-k split of a single problem (expand_count_kernel,
// expand_scan_kernel, expand_write_kernel): propagated states in, their first-fail children
// and fully fixed states out, in the order of the states.  ctr: [0] children written to
// `next`, [1] fully fixed states written to `units` (all levels so far), [2] nodes
// (branching or failed states), [3] failed states, [4] set when a buffer would overflow,
// [5] the level's first slot in `units`.  off: per state, its children and unit counts,
// then their exclusive prefix sums (count words).
struct ExpandArgs {
    const uint32_t *inst;
    const uint32_t *states;
    const int32_t *failed;
    int32_t count;
    uint32_t *next;
    int64_t next_cap;
    uint32_t *units;
    int64_t units_cap;
    unsigned long long *ctr;
    unsigned long long *off;
};

struct PropArgs {
    const uint32_t *inst;
    const uint32_t *din;
    uint32_t *dout;
    int32_t *failed;
    int32_t count;
    int32_t stage_words;
};

}  // namespace cubics
