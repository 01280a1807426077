// Host side of the CUBICS C ABI: model building and validation, encoding into the device
// layout of internal.h, workspace carving, and kernel launches (arxiv 1909.09213,
// Section 2.1: the host encodes the problem once and copies it to device memory; the search
// then runs on the device until its results are copied back).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/cubics.h"
#include "internal.h"

namespace cubics {
cudaError_t launch_search(int W, bool staged, int kind, const SearchArgs &A, int blocks,
                          int threads, size_t smem, cudaStream_t st);
cudaError_t occupancy_search(int W, bool staged, int kind, int threads, size_t smem,
                             int *blocks_per_sm);
cudaError_t launch_init_single(const SearchArgs &A, cudaStream_t st);
cudaError_t launch_init_batch(const SearchArgs &A, int teams, cudaStream_t st);
cudaError_t launch_propagate(int W, bool staged, const PropArgs &P, int blocks, int threads,
                             size_t smem, cudaStream_t st, bool block_per_node);
cudaError_t launch_expand(int W, const ExpandArgs &E, int blocks, cudaStream_t st);
cudaError_t probe_smem(void *out, cudaStream_t st, int sms, int reps, double *gbs);
cudaError_t mlp_pack(const uint16_t *params, uint32_t *packed, cudaStream_t st);
}  // namespace cubics

using namespace cubics;

namespace {

constexpr size_t SMEM_MAX = 232448;          // 227 KB dynamic shared memory per block
constexpr size_t ALIGN = 256;
constexpr int64_t BOUND_LIMIT = int64_t(1) << 30;

struct LinRow { std::vector<int32_t> coef, var; int32_t rhs; };
struct Table { int32_t x, y; std::vector<uint8_t> allowed; };   // size_x * size_y flags

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int natural_w(int span) {
    const int w = (span + 31) / 32;
    return w <= 1 ? 1 : w <= 2 ? 2 : w <= 4 ? 4 : 8;
}

struct DeviceInfo {
    int sms = 0;
    bool ok = false;
};

DeviceInfo device_info() {
    DeviceInfo d;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return d; }
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return d;
    }
    d.ok = true;
    return d;
}

struct Shape {
    int blocks = 0, warps = 0, lsm = 0, qcap = 0, stage_words = 0;
    int kind = KERN_PLAIN; // which search kernel (KERN_*)
    int mlp_words = 0;     // staged brancher weights (learned ordering)
    int feat_words = 0;    // per-warp feature tile (learned ordering)
    int list_words = 0;    // per-warp scheduled-table list (one-word tables)
    int hash_words = 0;    // per-warp deferred solution-hash buffer (register kernel)
    int warp_base = 0;     // shared-memory word where warp 0's area starts
    size_t smem = 0;
};

// Resources of one search launch.  R and depth are record words and stack levels per
// worker, cons the words of constraint data to stage in shared memory, nmax the largest
// number of variables (feature tile rows when `learned`); `reg`: every problem of the launch
// has FLAG_NE_REG (the register-held search kernel applies unless the learned brancher or
// logging is on).
int make_shape(const csp_tiling &t, int W, int R, int depth, int cons, bool batch, bool learned,
               bool logging, int nmax, int ntab, bool reg, Shape *s) {
    // the search kernels run one node per warp; a block per node is a propagate-only shape
    if (t.threads_per_node > 32) return CSP_EINVAL;
    s->kind = (learned || logging) ? KERN_EXT : reg ? KERN_REG : KERN_PLAIN;
    // one-word tables are revised from a per-warp list of the scheduled ones
    s->list_words = (W == 1 && ntab > 0) ? (ntab + 31) & ~31 : 0;
    s->warps = t.warps_per_block > 0 ? t.warps_per_block : 8;
    if (s->warps > 32) return CSP_EINVAL;
    s->mlp_words = learned ? CSP_MLP_PACKED_WORDS : 0;
    s->feat_words = learned ? ((nmax + 15) & ~15) * 8 : 0;
    s->hash_words = s->kind == KERN_REG ? HB_WORDS : 0;
    int lsm = t.smem_levels > 0 ? t.smem_levels : std::max(2, 6144 / R);
    lsm = std::max(2, std::min(lsm, depth));
    const int cons4 = (cons + 3) & ~3;
    auto bytes = [&](int l) {
        return ((size_t)s->warps * (l * R + WS_WORDS + s->feat_words + s->list_words + s->hash_words) +
                s->mlp_words) * 4;
    };
    // a power of two, so that a level's slot is its index masked: rounded up when the whole
    // stack was to fit (and still fits), down otherwise
    int p2 = 2;
    while (p2 < lsm) p2 <<= 1;
    const bool up = lsm == depth && bytes(p2) + (size_t)cons4 * 4 <= SMEM_MAX;
    lsm = (p2 == lsm || up) ? p2 : p2 >> 1;
    size_t smem = bytes(lsm);
    while (smem > SMEM_MAX && lsm > 2) smem = bytes(lsm >>= 1);
    if (smem > SMEM_MAX) return CSP_ETOOBIG;
    s->stage_words = (smem + (size_t)cons4 * 4 <= SMEM_MAX) ? cons4 : 0;
    s->warp_base = s->stage_words + s->mlp_words;
    s->smem = smem + (size_t)s->stage_words * 4;
    s->lsm = lsm;
    int q = t.queue_records > 0 ? t.queue_records : (batch ? 64 : 4096);
    if (q & (q - 1)) return CSP_EINVAL;
    s->qcap = q;
    // resident blocks per SM; 0 when a block of this many warps exceeds the kernel's
    // registers.  An explicit grid needs no device to be planned.
    int bps = 0;
    const cudaError_t oe =
        occupancy_search(W, s->stage_words > 0, s->kind, s->warps * 32, s->smem, &bps);
    if (oe != cudaSuccess) cudaGetLastError();
    if (oe == cudaSuccess && bps < 1) return CSP_EINVAL;
    if (t.blocks > 0) {
        s->blocks = t.blocks;
        return CSP_OK;
    }
    DeviceInfo di = device_info();
    if (!di.ok || oe != cudaSuccess) return CSP_ECUDA;
    s->blocks = di.sms * bps;
    return CSP_OK;
}

// The split depth of an all-solution search: 0 is the library's choice, 3 (measured on
// N-queens 12..16 with 4864 workers: 9-22x faster than one shared queue for trees of 10^5 -
// 10^7 nodes, the same for 2 * 10^8); -1 keeps one queue shared by every worker.
int split_depth_of(const csp_tiling &t) { return t.split_depth == 0 ? 3 : t.split_depth; }

// Two sibling nodes per warp, a half-warp each (threads_per_node 16, or 0: the library's
// choice): the register kernel (one-word int_ne, no learned brancher or logging) on problems
// of at most 16 variables, all-solution search.  1: pairs; 0: a warp per node; CSP_EINVAL:
// 16 asked where pairs do not apply.
int pairs_of(const csp_tiling &t, bool reg_kernel, int nmax, bool all) {
    const bool ok = reg_kernel && nmax <= 16 && all;
    if (t.threads_per_node == 16) return ok ? 1 : CSP_EINVAL;
    return (t.threads_per_node == 0 && ok) ? 1 : 0;
}

// Search levels a worker's stack holds.  Levels are nodes with an unfixed variable, so their
// tree depths are 0 .. n - 1 and rise from the bottom of the stack to the top: one per depth
// (n + 1 with a margin), or with pairs two per depth but the root's (a sibling's level
// waits below the level being searched), 2n - 1 (2n planned).
int stack_depth(int n, bool pairs) { return pairs ? 2 * n : n + 1; }

// carve consecutive 256-byte aligned regions
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, ALIGN);
        return o;
    }
};

}  // namespace

// ---------------------------------------------------------------------------- handle

// Layout of one single-problem workspace: the launch shape and the byte offset of every
// region.  Planning fills one of these without touching the handle, which takes it over
// only once the call that planned it can no longer fail for want of space.
struct Plan {
    Shape shape;
    int R = 0, depth = 0;
    int pairs = 0;                   // two sibling nodes per warp (register kernel)
    int W = 1;                       // words per domain of the search (csp_tiling.domain_words)
    size_t o_inst = 0, o_off = 0, o_g = 0, o_team = 0, o_qseq = 0, o_qrec = 0, o_spill = 0,
           o_sols = 0, o_mlp_params = 0, o_mlp_packed = 0;
    // all-solution search split at depth k into units solved by per-block teams
    bool split = false;
    int64_t ucap = 0;                // capacity of the unit buffers (states)
    size_t o_A = 0, o_B = 0, o_U = 0, o_failed = 0, o_scan = 0, o_ctr = 0, o_res = 0;
    size_t bytes = 0;
};

struct csp {
    int32_t n = 0;
    std::vector<int32_t> lo, hi;
    std::vector<std::vector<uint8_t>> present;       // per var, flags over lo..hi
    std::vector<int32_t> ne_x, ne_y, ne_c;
    std::vector<LinRow> lin;
    std::vector<std::vector<int32_t>> ad;
    std::vector<std::vector<int32_t>> adb;           // bounds-consistent alldifferent groups
    std::vector<Table> tab;
    int32_t lo0 = 0, W = 1;
    csp_tiling tiling{0, 0, 0, 0};
    int32_t brancher = CSP_BR_FIRST_FAIL;
    int32_t part = 0, nparts = 1;    // root children dealt round-robin across ranks
    // device binding
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;   // ev2: before a split's search
    // last upload
    bool uploaded = false;
    int32_t up_mode = -1;
    int64_t up_cap = 0;
    std::vector<uint32_t> block;
    uint32_t *pin_block = nullptr;   // pinned host staging of the encoded problem
    size_t pin_words = 0;
    GState *pin_g = nullptr;         // pinned host copy of the launch counters
    Plan plan;                       // workspace layout of the last upload
    uint64_t split_nodes = 0, split_fails = 0;   // nodes of the levels a split expanded
    int64_t split_units = 0;
    std::vector<uint16_t> mlp_params;    // learned brancher weights (bf16)
    csp_stats_t stats{};
};

namespace {

int var_ok(const csp *h, int32_t v) { return h && v >= 0 && v < h->n; }

void invalidate(csp *h) { h->uploaded = false; }

// Encode the model with W words per domain (W >= the model's own W).
void encode(const csp *h, int W, std::vector<uint32_t> &B) {
    const int n = h->n, S = n * W, NW = (n + 31) / 32;
    const int lo0 = h->lo0;
    const int span = 32 * W;
    B.assign(HDR_WORDS, 0u);
    auto put = [&](uint32_t v) { B.push_back(v); };
    auto align4 = [&]() { while (B.size() & 3) B.push_back(0u); };
    uint32_t flags = 0;
    // unary ne
    std::vector<uint32_t> un;
    std::vector<std::vector<uint32_t>> adj(n);
    size_t n_ne = 0;
    for (size_t k = 0; k < h->ne_x.size(); ++k) {
        const int x = h->ne_x[k], y = h->ne_y[k];
        const int64_t c = h->ne_c[k];
        n_ne++;
        if (y < 0) {
            const int64_t bit = c - lo0;
            if (bit >= 0 && bit < span) un.push_back((uint32_t)x | ((uint32_t)bit << 16));
        } else if (c > -span && c < span) {
            adj[y].push_back((uint32_t)x | ((uint32_t)(uint16_t)(int16_t)c << 16));
            adj[x].push_back((uint32_t)y | ((uint32_t)(uint16_t)(int16_t)(-c) << 16));
        }
    }
    B[H_N] = n; B[H_W] = W; B[H_LO0] = (uint32_t)lo0; B[H_S] = S; B[H_NW] = NW;
    B[H_N_NE] = (uint32_t)n_ne;
    B[H_N_UN] = (uint32_t)un.size();
    B[H_OFF_UN] = (uint32_t)B.size();
    for (uint32_t u : un) put(u);
    B[H_OFF_ADJ_START] = (uint32_t)B.size();
    uint32_t acc = 0;
    for (int v = 0; v < n; ++v) { put(acc); acc += (uint32_t)adj[v].size(); }
    put(acc);
    B[H_OFF_ADJ] = (uint32_t)B.size();
    for (int v = 0; v < n; ++v) for (uint32_t e : adj[v]) put(e);
    // lin rows (already merged at post time)
    const int nl = (int)h->lin.size();
    B[H_N_LIN] = nl;
    B[H_OFF_LIN_ROW] = (uint32_t)B.size();
    uint32_t t0 = 0;
    for (const LinRow &r : h->lin) {
        put(t0); put((uint32_t)r.coef.size()); put((uint32_t)r.rhs);
        t0 += (uint32_t)r.coef.size();
        if (r.coef.empty() && r.rhs < 0) flags |= FLAG_TRIVIAL_FAIL;
    }
    B[H_OFF_LIN_TERM] = (uint32_t)B.size();
    for (const LinRow &r : h->lin)
        for (size_t t = 0; t < r.coef.size(); ++t) { put((uint32_t)r.coef[t]); put((uint32_t)r.var[t]); }
    const int lmw = (nl + 31) / 32;
    B[H_LIN_MW] = lmw;
    B[H_OFF_LIN_MASK] = (uint32_t)B.size();
    {
        std::vector<uint32_t> m((size_t)n * lmw, 0u);
        for (int r = 0; r < nl; ++r)
            for (int32_t v : h->lin[r].var) m[(size_t)v * lmw + r / 32] |= 1u << (r % 32);
        for (uint32_t w : m) put(w);
    }
    // alldiff
    const int na = (int)h->ad.size();
    B[H_N_AD] = na;
    B[H_OFF_AD_ROW] = (uint32_t)B.size();
    uint32_t m0 = 0;
    for (const auto &g : h->ad) { put(m0); put((uint32_t)g.size()); m0 += (uint32_t)g.size(); }
    B[H_OFF_AD_MEM] = (uint32_t)B.size();
    for (const auto &g : h->ad) for (int32_t v : g) put((uint32_t)v);
    const int amw = (na + 31) / 32;
    B[H_AD_MW] = amw;
    B[H_OFF_AD_MASK] = (uint32_t)B.size();
    {
        std::vector<uint32_t> m((size_t)n * amw, 0u);
        for (int g = 0; g < na; ++g)
            for (int32_t v : h->ad[g]) m[(size_t)v * amw + g / 32] |= 1u << (g % 32);
        for (uint32_t w : m) put(w);
    }
    // bounds-consistent alldifferent groups (same layout as the alldiff ones)
    const int nb = (int)h->adb.size();
    B[H_N_ADB] = nb;
    B[H_OFF_ADB_ROW] = (uint32_t)B.size();
    uint32_t b0 = 0;
    for (const auto &g : h->adb) { put(b0); put((uint32_t)g.size()); b0 += (uint32_t)g.size(); }
    B[H_OFF_ADB_MEM] = (uint32_t)B.size();
    for (const auto &g : h->adb) for (int32_t v : g) put((uint32_t)v);
    const int bmw = (nb + 31) / 32;
    B[H_ADB_MW] = bmw;
    B[H_OFF_ADB_MASK] = (uint32_t)B.size();
    {
        std::vector<uint32_t> m((size_t)n * bmw, 0u);
        for (int g = 0; g < nb; ++g)
            for (int32_t v : h->adb[g]) m[(size_t)v * bmw + g / 32] |= 1u << (g % 32);
        for (uint32_t w : m) put(w);
    }
    // tables: 4-word entries, then the R/C matrices (32*W rows of W words each)
    const int nt = (int)h->tab.size();
    B[H_N_TAB] = nt;
    B[H_OFF_TAB] = (uint32_t)B.size();
    const size_t tab_hdr = B.size();
    for (int t = 0; t < nt; ++t) { put(0); put(0); put(0); put(0); }
    for (int t = 0; t < nt; ++t) {
        const Table &T = h->tab[t];
        const int sx = h->hi[T.x] - h->lo[T.x] + 1, sy = h->hi[T.y] - h->lo[T.y] + 1;
        const int ox = h->lo[T.x] - lo0, oy = h->lo[T.y] - lo0;
        align4();
        const size_t offR = B.size();
        B.resize(offR + (size_t)2 * span * W, 0u);
        const size_t offC = offR + (size_t)span * W;
        for (int a = 0; a < sx; ++a)
            for (int b = 0; b < sy; ++b)
                if (T.allowed[(size_t)a * sy + b]) {
                    const int ba = ox + a, bb = oy + b;
                    B[offR + (size_t)ba * W + bb / 32] |= 1u << (bb % 32);
                    B[offC + (size_t)bb * W + ba / 32] |= 1u << (ba % 32);
                }
        B[tab_hdr + 4 * t] = (uint32_t)T.x;
        B[tab_hdr + 4 * t + 1] = (uint32_t)T.y;
        B[tab_hdr + 4 * t + 2] = (uint32_t)offR;
        B[tab_hdr + 4 * t + 3] = (uint32_t)offC;
    }
    // static data for the learned brancher's features, and neighbour lists
    {
        std::vector<int> deg(n, 0), kne(n, 0), klin(n, 0), kad(n, 0), ktab(n, 0);
        std::vector<double> tight(n, 0.0);
        // neighbour sets as a bit matrix (a row of n bits per variable): long rows, such as
        // an objective bound over every variable, cost one bit per pair
        const size_t nw64 = ((size_t)n + 63) / 64;
        std::vector<uint64_t> nbm((size_t)n * nw64, 0ull);
        auto link = [&](int a, int b) {
            if (a != b) {
                nbm[(size_t)a * nw64 + b / 64] |= 1ull << (b % 64);
                nbm[(size_t)b * nw64 + a / 64] |= 1ull << (a % 64);
            }
        };
        for (size_t k = 0; k < h->ne_x.size(); ++k) {
            const int x = h->ne_x[k], y = h->ne_y[k];
            deg[x]++; kne[x]++;
            if (y >= 0 && y != x) { deg[y]++; kne[y]++; link(x, y); }
        }
        for (const LinRow &r : h->lin) {
            for (int32_t v : r.var) { deg[v]++; klin[v]++; }
            for (size_t a = 0; a < r.var.size(); ++a)
                for (size_t b = a + 1; b < r.var.size(); ++b) link(r.var[a], r.var[b]);
        }
        for (const auto &g : h->adb) {     // counted with the alldifferent groups
            for (int32_t v : g) { deg[v]++; kad[v]++; }
            for (size_t a = 0; a < g.size(); ++a)
                for (size_t b = a + 1; b < g.size(); ++b) link(g[a], g[b]);
        }
        for (const auto &g : h->ad) {
            for (int32_t v : g) { deg[v]++; kad[v]++; }
            for (size_t a = 0; a < g.size(); ++a)
                for (size_t b = a + 1; b < g.size(); ++b) link(g[a], g[b]);
        }
        for (const Table &T : h->tab) {
            size_t allowed = 0;
            for (uint8_t f : T.allowed) allowed += f;
            const double forb = 1.0 - (double)allowed / (double)std::max<size_t>(1, T.allowed.size());
            deg[T.x]++; ktab[T.x]++; tight[T.x] += forb;
            deg[T.y]++; ktab[T.y]++; tight[T.y] += forb;
            link(T.x, T.y);
        }
        int maxdeg = 1;
        for (int v = 0; v < n; ++v) maxdeg = std::max(maxdeg, deg[v]);
        B[H_MAXDEG] = (uint32_t)maxdeg;
        B[H_OFF_VFEAT] = (uint32_t)B.size();
        for (int v = 0; v < n; ++v) {
            const float t = ktab[v] ? (float)(tight[v] / ktab[v]) : 0.f;
            uint32_t tb;
            std::memcpy(&tb, &t, 4);
            put((uint32_t)(h->lo[v] - lo0)); put((uint32_t)(h->hi[v] - h->lo[v] + 1));
            put((uint32_t)deg[v]); put((uint32_t)kne[v]); put((uint32_t)klin[v]);
            put((uint32_t)kad[v]); put((uint32_t)ktab[v]); put(tb);
        }
        B[H_OFF_NB_START] = (uint32_t)B.size();
        uint32_t s0 = 0;
        for (int v = 0; v < n; ++v) {
            put(s0);
            for (size_t k = 0; k < nw64; ++k) s0 += (uint32_t)__builtin_popcountll(nbm[(size_t)v * nw64 + k]);
        }
        put(s0);
        B[H_OFF_NB] = (uint32_t)B.size();
        for (int v = 0; v < n; ++v)                    // ascending neighbour indices
            for (size_t k = 0; k < nw64; ++k)
                for (uint64_t w = nbm[(size_t)v * nw64 + k]; w; w &= w - 1)
                    put((uint32_t)(k * 64 + (size_t)__builtin_ctzll(w)));
    }
    // int_ne offset masks for a search that keeps one-word domains in registers
    const bool ne_only = h->lin.empty() && h->ad.empty() && h->tab.empty() && h->adb.empty();
    if (ne_only && W == 1 && n <= 32) {
        flags |= FLAG_NE_REG;
        while (B.size() & 1) B.push_back(0u);                 // 8-byte aligned pairs
        const size_t nm = B.size();
        B[H_OFF_NEMASK] = (uint32_t)nm;
        B.resize(nm + (size_t)2 * 32 * n, 0u);
        for (int v = 0; v < n; ++v)
            for (uint32_t e : adj[v]) {                        // fixing v removes val + off from t
                const int t = (int)(e & 0xffffu), off = (int)(int16_t)(e >> 16);
                if (off < -31 || off > 31) continue;
                const int bit = off + 31;
                B[nm + 2 * ((size_t)v * 32 + t) + (bit >> 5)] |= 1u << (bit & 31);
            }
    }
    align4();
    B[H_CONS_WORDS] = (uint32_t)B.size();
    B[H_OFF_ROOT] = (uint32_t)B.size();
    const size_t root = B.size();
    B.resize(root + (size_t)S, 0u);
    for (int i = 0; i < n; ++i) {
        const int o = h->lo[i] - lo0;
        for (int k = 0; k <= h->hi[i] - h->lo[i]; ++k)
            if (h->present[i][k]) B[root + (size_t)i * W + (o + k) / 32] |= 1u << ((o + k) % 32);
    }
    while (B.size() & 63) B.push_back(0u);
    B[H_TOTAL] = (uint32_t)B.size();
    B[H_R] = (uint32_t)record_words(S, W);
    if (ne_only) flags |= FLAG_NE_ONLY;
    B[H_FLAGS] = flags;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CSP_OK;
    cudaGetLastError();
    return CSP_ECUDA;
}

// Layout of a single-problem workspace for mode/cap under the current tiling; `blk`
// receives the encoded problem.  The handle is not modified.
int plan_single(const csp *h, int32_t mode, int64_t cap, Plan *P, std::vector<uint32_t> *blk,
                bool allow_split = true) {
    std::vector<uint32_t> local;
    std::vector<uint32_t> &B = blk ? *blk : local;
    // a search may run with wider domains than the problem's own (the tuner's width axis);
    // propagation keeps the problem's layout
    const int W = mode == CSP_PROPAGATE ? h->W : std::max(h->W, (int)h->tiling.domain_words);
    encode(h, W, B);
    Plan p;
    Carver c;
    p.o_inst = c.take(B.size() * 4);
    p.o_off = c.take(sizeof(int64_t));
    if (mode == CSP_PROPAGATE) {
        const size_t sw = (size_t)h->n * h->W * 4;
        p.o_qseq = c.take(sw * (size_t)cap);     // dom_in
        p.o_qrec = c.take(sw * (size_t)cap);     // dom_out
        p.o_sols = c.take(4 * (size_t)cap);      // failed
        p.bytes = c.off;
        *P = p;
        return CSP_OK;
    }
    const int R = record_words(h->n * W, W);
    const bool learned = h->brancher == CSP_BR_LEARNED;
    const int pairs = pairs_of(h->tiling, (B[H_FLAGS] & FLAG_NE_REG) != 0 && !learned, h->n,
                               mode == CSP_ALL);
    if (pairs < 0) return pairs;
    const int depth = stack_depth(h->n, pairs > 0);
    // the device expansion of the first levels branches first-fail: a learned ordering
    // searches the whole tree with one shared queue
    p.split = allow_split && mode == CSP_ALL && split_depth_of(h->tiling) > 0 && h->nparts == 1 &&
              !learned;
    int rc = make_shape(h->tiling, W, R, depth, (int)B[H_CONS_WORDS], p.split, learned, false,
                        h->n, (int)B[H_N_TAB], (B[H_FLAGS] & FLAG_NE_REG) != 0, &p.shape);
    if (rc) return rc;
    const Shape &s = p.shape;
    p.R = R;
    p.depth = depth;
    p.pairs = pairs;
    p.W = W;
    if (p.split) {
        // per-block teams (one queue each) over the units, the level buffers and the units
        const size_t S4 = (size_t)h->n * W * 4;
        p.ucap = std::max<int64_t>(1024, std::min<int64_t>(1 << 16, (int64_t)((32u << 20) / S4)));
        p.o_off = c.take((size_t)(2 * p.ucap) * 8);              // zero block offsets
        p.o_g = c.take(sizeof(GState));
        p.o_team = c.take((size_t)s.blocks * sizeof(Team));
        p.o_qseq = c.take((size_t)s.blocks * s.qcap * 4);
        p.o_qrec = c.take((size_t)s.blocks * s.qcap * R * 4);
        p.o_spill = c.take((size_t)s.blocks * s.warps * depth * R * 4);
        p.o_sols = c.take((size_t)std::max<int64_t>(cap, 1) * h->n * 4);
        p.o_res = c.take((size_t)(2 * p.ucap) * sizeof(InstResult));
        p.o_A = c.take((size_t)(2 * p.ucap) * S4);
        p.o_B = c.take((size_t)(2 * p.ucap) * S4);
        p.o_U = c.take((size_t)p.ucap * S4);
        p.o_failed = c.take((size_t)(2 * p.ucap) * 4);
        p.o_scan = c.take((size_t)(2 * p.ucap) * 8);
        p.o_ctr = c.take(8 * 8);
        p.bytes = c.off;
        *P = p;
        return CSP_OK;
    }
    p.o_g = c.take(sizeof(GState));
    p.o_team = c.take(sizeof(Team));
    p.o_qseq = c.take((size_t)s.qcap * 4);
    p.o_qrec = c.take((size_t)s.qcap * R * 4);
    p.o_spill = c.take((size_t)s.blocks * s.warps * depth * R * 4);
    p.o_sols = c.take((size_t)std::max<int64_t>(cap, 1) * h->n * 4);
    p.o_mlp_params = c.take(learned ? CSP_MLP_PARAMS * 2 : 0);
    p.o_mlp_packed = c.take(learned ? CSP_MLP_PACKED_WORDS * 4 : 0);
    p.bytes = c.off;
    *P = p;
    return CSP_OK;
}

// the brancher's bf16 parameters into the workspace, then their fragment-ordered copy
cudaError_t upload_mlp(const std::vector<uint16_t> &params, uint8_t *ws, size_t o_params,
                       size_t o_packed, cudaStream_t st) {
    // both regions follow the problem's block (offset 0): a plan without them has none
    if (o_params == 0 || o_packed == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(ws + o_params, params.data(), params.size() * 2,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = mlp_pack((const uint16_t *)(ws + o_params), (uint32_t *)(ws + o_packed), st);
    return e;
}

void set_learned_args(SearchArgs &A, const Shape &s, bool learned, const uint8_t *ws, size_t o_packed) {
    A.mlp = learned ? (const uint32_t *)(ws + o_packed) : nullptr;
    A.mlp_off = learned ? s.stage_words : -1;
    A.feat_words = s.feat_words;
    A.list_words = s.list_words;
    A.hash_words = s.hash_words;
    A.warp_base = s.warp_base;
}

SearchArgs single_args(const csp *h, const Plan &P, uint8_t *w, int32_t mode, int64_t cap,
                       const csp_limits *lim) {
    SearchArgs A{};
    A.arena = (const uint32_t *)(w + P.o_inst);
    A.inst_off = (const int64_t *)(w + P.o_off);
    A.sol_off = nullptr;
    A.n_inst = 1;
    A.mode = mode;
    A.batch = 0;
    A.lsm = P.shape.lsm;
    A.rmax = P.R;
    A.depth = P.depth;
    A.pairs = P.pairs;
    A.stage_words = P.shape.stage_words;
    A.qmask = P.shape.qcap - 1;
    A.flags = lim ? lim->flags : 0;
    A.warps = P.shape.warps;
    A.g = (GState *)(w + P.o_g);
    A.teams = (Team *)(w + P.o_team);
    A.qseq = (uint32_t *)(w + P.o_qseq);
    A.qrec = (uint32_t *)(w + P.o_qrec);
    A.spill = (uint32_t *)(w + P.o_spill);
    A.sols = (int32_t *)(w + P.o_sols);
    A.cap = mode == CSP_FIRST ? 1 : cap;
    A.results = nullptr;
    A.node_limit = lim ? lim->node_limit : 0;
    A.deadline_ns = lim ? lim->time_limit_ns : 0;
    A.wait_limit_ns = (lim && lim->wait_limit_ns > 0) ? lim->wait_limit_ns : 60000000000LL;
    set_learned_args(A, P.shape, h->brancher == CSP_BR_LEARNED, w, P.o_mlp_packed);
    A.log_extra = 0;
    A.log_sample = 1;
    A.logbuf = nullptr;
    A.log_count = nullptr;
    A.log_cap = 0;
    A.part = h->part;
    A.nparts = h->nparts;
    return A;
}

void fill_stats(csp_stats_t *s, const GState &g, int64_t stored) {
    s->nodes = g.nodes;
    s->fails = g.fails;
    s->solutions = g.solutions;
    s->sol_hash_sum = g.hsum;
    s->sol_hash_xor = g.hxor;
    s->prop_evals = g.evals;
    s->steals = g.steals;
    s->spills = g.spills;
    s->max_depth = g.max_depth;
    s->stored = stored;
    s->wait_ns = g.wait_ns;
    s->rounds = g.rounds;
}

}  // namespace

// ---------------------------------------------------------------------------- model calls

extern "C" {

int csp_create(csp_t **out, int32_t n_vars, const int32_t *lo, const int32_t *hi) {
    if (!out || !lo || !hi || n_vars < 1) return CSP_EINVAL;
    if (n_vars > MAX_VARS) return CSP_ETOOBIG;
    int64_t mn = INT32_MAX, mx = INT32_MIN;
    for (int i = 0; i < n_vars; ++i) {
        if (hi[i] < lo[i]) return CSP_EINVAL;
        mn = std::min<int64_t>(mn, lo[i]);
        mx = std::max<int64_t>(mx, hi[i]);
    }
    if (mx - mn + 1 > 256) return CSP_ETOOBIG;
    csp *h = new csp();
    h->n = n_vars;
    h->lo.assign(lo, lo + n_vars);
    h->hi.assign(hi, hi + n_vars);
    h->present.resize(n_vars);
    for (int i = 0; i < n_vars; ++i) h->present[i].assign((size_t)(hi[i] - lo[i] + 1), 1);
    h->lo0 = (int32_t)mn;
    h->W = natural_w((int)(mx - mn + 1));
    *out = h;
    return CSP_OK;
}

int csp_remove_value(csp_t *h, int32_t var, int32_t value) {
    if (!var_ok(h, var)) return CSP_EINVAL;
    if (value >= h->lo[var] && value <= h->hi[var]) h->present[var][value - h->lo[var]] = 0;
    invalidate(h);
    return CSP_OK;
}

int csp_post_int_ne(csp_t *h, int32_t x, int32_t y, int32_t c) {
    if (!var_ok(h, x) || (y >= 0 && !var_ok(h, y)) || !h) return CSP_EINVAL;
    h->ne_x.push_back(x);
    h->ne_y.push_back(y < 0 ? -1 : y);
    h->ne_c.push_back(c);
    invalidate(h);
    return CSP_OK;
}

int csp_post_int_lin_le(csp_t *h, int32_t k, const int32_t *coef, const int32_t *vars,
                        int32_t rhs) {
    if (!h || k < 0 || (k > 0 && (!coef || !vars))) return CSP_EINVAL;
    std::map<int32_t, int64_t> merged;
    std::vector<int32_t> order;
    for (int t = 0; t < k; ++t) {
        if (!var_ok(h, vars[t])) return CSP_EINVAL;
        if (!merged.count(vars[t])) order.push_back(vars[t]);
        merged[vars[t]] += coef[t];
    }
    LinRow r;
    int64_t bound = std::abs((int64_t)rhs);
    for (int32_t v : order) {
        const int64_t a = merged[v];
        if (a == 0) continue;
        const int64_t mag = std::max(std::abs((int64_t)h->lo[v]), std::abs((int64_t)h->hi[v]));
        const int64_t win = std::max(std::abs((int64_t)h->lo0), std::abs((int64_t)h->lo0 + 255));
        bound += std::abs(a) * std::max(mag, win);
        if (bound >= BOUND_LIMIT) return CSP_ETOOBIG;
        r.coef.push_back((int32_t)a);
        r.var.push_back(v);
    }
    r.rhs = rhs;
    h->lin.push_back(r);
    invalidate(h);
    return CSP_OK;
}

int csp_post_alldiff(csp_t *h, int32_t k, const int32_t *vars) {
    if (!h || k < 0 || (k > 0 && !vars)) return CSP_EINVAL;
    std::vector<int32_t> g(vars, vars + k);
    for (int32_t v : g) if (!var_ok(h, v)) return CSP_EINVAL;
    std::vector<int32_t> s = g;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return CSP_EINVAL;
    h->ad.push_back(g);
    invalidate(h);
    return CSP_OK;
}

int csp_post_alldiff_bc(csp_t *h, int32_t k, const int32_t *vars) {
    if (!h || k < 0 || (k > 0 && !vars)) return CSP_EINVAL;
    if (k > ADB_MAX) return CSP_ETOOBIG;
    std::vector<int32_t> g(vars, vars + k);
    for (int32_t v : g) if (!var_ok(h, v)) return CSP_EINVAL;
    std::vector<int32_t> s = g;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return CSP_EINVAL;
    h->adb.push_back(g);
    invalidate(h);
    return CSP_OK;
}

int csp_post_table(csp_t *h, int32_t x, int32_t y, const uint32_t *allowed, int32_t row_words) {
    if (!var_ok(h, x) || !var_ok(h, y) || x == y || !allowed) return CSP_EINVAL;
    const int sx = h->hi[x] - h->lo[x] + 1, sy = h->hi[y] - h->lo[y] + 1;
    if (row_words < (sy + 31) / 32) return CSP_EINVAL;
    Table T;
    T.x = x;
    T.y = y;
    T.allowed.assign((size_t)sx * sy, 0);
    for (int a = 0; a < sx; ++a)
        for (int b = 0; b < sy; ++b)
            T.allowed[(size_t)a * sy + b] = (allowed[(size_t)a * row_words + b / 32] >> (b % 32)) & 1u;
    h->tab.push_back(std::move(T));
    invalidate(h);
    return CSP_OK;
}

int csp_root_domains(const csp_t *h, uint32_t *out) {
    if (!h || !out) return CSP_EINVAL;
    const int W = h->W;
    for (int i = 0; i < h->n; ++i) {
        for (int k = 0; k < W; ++k) out[(size_t)i * W + k] = 0u;
        for (int32_t v = h->lo[i]; v <= h->hi[i]; ++v) {
            if (!h->present[i][v - h->lo[i]]) continue;
            const int b = v - h->lo0;
            out[(size_t)i * W + b / 32] |= 1u << (b % 32);
        }
    }
    return CSP_OK;
}

int csp_clone(const csp_t *src, csp_t **out) {
    if (!src || !out) return CSP_EINVAL;
    csp *h = new csp();
    h->n = src->n;
    h->lo = src->lo;
    h->hi = src->hi;
    h->present = src->present;
    h->ne_x = src->ne_x;
    h->ne_y = src->ne_y;
    h->ne_c = src->ne_c;
    h->lin = src->lin;
    h->ad = src->ad;
    h->adb = src->adb;
    h->tab = src->tab;
    h->lo0 = src->lo0;
    h->W = src->W;
    h->tiling = src->tiling;
    h->brancher = src->brancher;
    h->mlp_params = src->mlp_params;
    h->part = src->part;
    h->nparts = src->nparts;
    *out = h;
    return CSP_OK;
}

int csp_fix_values(csp_t *h, int32_t count, const int32_t *vars, const int32_t *values) {
    if (!h || count < 0 || (count > 0 && (!vars || !values))) return CSP_EINVAL;
    for (int t = 0; t < count; ++t)
        if (!var_ok(h, vars[t])) return CSP_EINVAL;
    for (int t = 0; t < count; ++t) {
        const int32_t v = vars[t], val = values[t];
        std::vector<uint8_t> &p = h->present[v];
        const bool had = val >= h->lo[v] && val <= h->hi[v] && p[val - h->lo[v]];
        std::fill(p.begin(), p.end(), (uint8_t)0);
        if (had) p[val - h->lo[v]] = 1;
    }
    invalidate(h);
    return CSP_OK;
}

int csp_layout(const csp_t *h, int32_t *n, int32_t *W, int32_t *lo0) {
    if (!h) return CSP_EINVAL;
    if (n) *n = h->n;
    if (W) *W = h->W;
    if (lo0) *lo0 = h->lo0;
    return CSP_OK;
}

// queue capacity a power of two; threads per node 0 or a multiple of 32 up to 1024
static bool tiling_ok(const csp_tiling &t) {
    const int tp = t.threads_per_node;
    const int dw = t.domain_words;
    return !(t.queue_records & (t.queue_records - 1)) && tp >= 0 && tp <= 1024 &&
           (tp % 32 == 0 || tp == 16) && t.split_depth >= -1 && t.split_depth <= 8 &&
           (dw == 0 || dw == 1 || dw == 2 || dw == 4 || dw == 8);
}

int csp_set_tiling(csp_t *h, const csp_tiling *t) {
    if (!h) return CSP_EINVAL;
    const csp_tiling nt = t ? *t : csp_tiling{0, 0, 0, 0, 0, 0, 0};
    if (!tiling_ok(nt)) return CSP_EINVAL;
    h->tiling = nt;
    invalidate(h);
    return CSP_OK;
}

int csp_set_partition(csp_t *h, int32_t part, int32_t nparts) {
    if (!h || nparts < 1 || part < 0 || part >= nparts) return CSP_EINVAL;
    h->part = part;
    h->nparts = nparts;
    return CSP_OK;
}

int csp_set_brancher(csp_t *h, int32_t kind, const uint16_t *bf16_weights) {
    if (!h || (kind != CSP_BR_FIRST_FAIL && kind != CSP_BR_LEARNED)) return CSP_EINVAL;
    if (kind == CSP_BR_LEARNED) {
        if (bf16_weights) h->mlp_params.assign(bf16_weights, bf16_weights + CSP_MLP_PARAMS);
        if (h->mlp_params.size() != (size_t)CSP_MLP_PARAMS) return CSP_EINVAL;
    }
    h->brancher = kind;
    invalidate(h);
    return CSP_OK;
}

int csp_workspace_bytes(const csp_t *hc, int32_t mode, int64_t cap, size_t *bytes) {
    if (!hc || !bytes || mode < 0 || mode > 2 || cap < 0 || cap > INT32_MAX) return CSP_EINVAL;
    Plan P;
    const int rc = plan_single(hc, mode, cap, &P, nullptr);
    if (rc) return rc;
    *bytes = P.bytes;
    return CSP_OK;
}

int csp_bind(csp_t *h, void *dev, size_t bytes, void *cuda_stream) {
    if (!h || !dev || ((uintptr_t)dev % ALIGN)) return CSP_EINVAL;
    if (!h->ev0) {
        if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
            cudaEventCreate(&h->ev2) != cudaSuccess) {
            cudaGetLastError();
            return CSP_ECUDA;
        }
    }
    h->ws = (uint8_t *)dev;
    h->ws_bytes = bytes;
    h->stream = (cudaStream_t)cuda_stream;
    invalidate(h);
    return CSP_OK;
}

int csp_upload(csp_t *h, int32_t mode, int64_t cap) {
    if (!h || mode < 0 || mode > 1 || cap < 0 || cap > INT32_MAX) return CSP_EINVAL;
    if (!h->ws) return CSP_ESTATE;
    Plan P;
    std::vector<uint32_t> B;
    int rc = plan_single(h, mode, cap, &P, &B);
    if (rc) return rc;
    if (P.bytes > h->ws_bytes) return CSP_ENOMEM;
    // stage through pinned host memory: the encoded problem, then its block offset (0)
    const size_t words = B.size() + 2;
    if (h->pin_words < words) {
        if (h->pin_block) cudaFreeHost(h->pin_block);
        h->pin_block = nullptr;
        h->pin_words = 0;
        if (cudaMallocHost(&h->pin_block, words * 4) != cudaSuccess) {
            cudaGetLastError();
            return CSP_ECUDA;
        }
        h->pin_words = words;
    }
    if (!h->pin_g && cudaMallocHost(&h->pin_g, sizeof(GState)) != cudaSuccess) {
        cudaGetLastError();
        h->pin_g = nullptr;
        return CSP_ECUDA;
    }
    // from here on the workspace is overwritten: the previous upload is no longer valid
    h->uploaded = false;
    h->plan = P;
    h->block.swap(B);
    std::memcpy(h->pin_block, h->block.data(), h->block.size() * 4);
    h->pin_block[h->block.size()] = 0u;
    h->pin_block[h->block.size() + 1] = 0u;
    cudaError_t e = cudaMemcpyAsync(h->ws + P.o_inst, h->pin_block, h->block.size() * 4,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws + P.o_off, h->pin_block + h->block.size(), sizeof(int64_t),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->brancher == CSP_BR_LEARNED)
        e = upload_mlp(h->mlp_params, h->ws, P.o_mlp_params, P.o_mlp_packed, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->stats.h2d_bytes = (int64_t)h->block.size() * 4 + (int64_t)sizeof(int64_t) +
                         (h->brancher == CSP_BR_LEARNED ? CSP_MLP_PARAMS * 2 : 0);
    h->uploaded = true;
    h->up_mode = mode;
    h->up_cap = cap;
    return CSP_OK;
}

// The all-solution search split at depth k (csp_tiling.split_depth): the root is copied to
// level buffer A; each of the first k levels is propagated in place and expanded into B
// (children) and U (states with every variable fixed), both in the order of their parents
// (the units come out in depth-first order at every run), the counters read back after each
// level; an expansion that would overflow a buffer is undone and its (propagated) level
// becomes the units.  The units (A's states, then U's) are then solved as a batch whose
// instances share the problem's block and take their roots from A, each block's warps
// sharing one unit through the block's queue.  Waits for the device between levels.
static cudaError_t split_launch(csp *h, const csp_limits *lim) {
    const Plan &P = h->plan;
    const cudaStream_t st = h->stream;
    uint8_t *w = h->ws;
    const int n = h->n, W = P.W, S = n * W;
    const size_t S4 = (size_t)S * 4;
    const uint32_t *blk = (const uint32_t *)(w + P.o_inst);
    uint8_t *A = w + P.o_A, *Bf = w + P.o_B;
    unsigned long long *ctr = (unsigned long long *)(w + P.o_ctr);
    // the launch's device time includes the level expansions (and the waits between them)
    cudaError_t e = cudaEventRecord(h->ev0, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(A, w + P.o_inst + (size_t)h->block[H_OFF_ROOT] * 4, S4,
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 8 * 8, st);
    // propagation shape: a warp per state, as many warps per block as fit
    const int cons4 = ((int)h->block[H_CONS_WORDS] + 3) & ~3;
    const size_t per_state = (size_t)(((S + 3) & ~3) + 64) * 4;
    int pw = 8;
    while (pw > 1 && per_state * pw > SMEM_MAX) --pw;
    PropArgs PA{};
    PA.inst = blk;
    PA.failed = (int32_t *)(w + P.o_failed);
    const size_t psm0 = per_state * pw;
    PA.stage_words = (psm0 + (size_t)cons4 * 4 <= SMEM_MAX) ? cons4 : 0;
    const size_t psm = psm0 + (size_t)PA.stage_words * 4;
    if (psm > SMEM_MAX) return cudaErrorInvalidValue;
    unsigned long long prev[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cur[8];
    int64_t count = 1;
    for (int d = 0; d < split_depth_of(h->tiling) && e == cudaSuccess && count > 0; ++d) {
        PA.din = (const uint32_t *)A;
        PA.dout = (uint32_t *)A;
        PA.count = (int32_t)count;
        const int pblocks = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (count + pw - 1) / pw));
        e = launch_propagate(W, PA.stage_words > 0, PA, pblocks, pw * 32, psm, st, false);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 8, st);                // children
        if (e == cudaSuccess) e = cudaMemsetAsync(ctr + 4, 0, 8, st);            // overflow
        ExpandArgs E{};
        E.inst = blk;
        E.states = (const uint32_t *)A;
        E.failed = PA.failed;
        E.count = (int32_t)count;
        E.next = (uint32_t *)Bf;
        E.next_cap = P.ucap;
        E.units = (uint32_t *)(w + P.o_U);
        E.units_cap = P.ucap;
        E.ctr = ctr;
        E.off = (unsigned long long *)(w + P.o_scan);
        const int eblocks = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (count + 7) / 8));
        if (e == cudaSuccess) e = launch_expand(W, E, eblocks, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cur, ctr, sizeof(cur), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (cur[4]) {                       // overflow: this level's states become the units
            e = cudaMemcpyAsync(ctr, prev, sizeof(prev), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            break;
        }
        std::memcpy(prev, cur, sizeof(prev));
        std::swap(A, Bf);
        count = (int64_t)cur[0];
    }
    if (e != cudaSuccess) return e;
    // the units: A's states, then the fully fixed states of U
    const int64_t nu = (int64_t)prev[1];
    if (nu > 0) e = cudaMemcpyAsync(A + (size_t)count * S4, w + P.o_U, (size_t)nu * S4,
                                    cudaMemcpyDeviceToDevice, st);
    const int64_t units = count + nu;
    h->split_nodes = prev[2];
    h->split_fails = prev[3];
    h->split_units = units;
    if (e == cudaSuccess) e = cudaMemsetAsync(w + P.o_g, 0, sizeof(GState), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w + P.o_team, 0, (size_t)P.shape.blocks * sizeof(Team), st);
    if (e == cudaSuccess && units > 0)
        e = cudaMemsetAsync(w + P.o_off, 0, (size_t)units * 8, st);
    if (e == cudaSuccess && units > 0)
        e = cudaMemsetAsync(w + P.o_res, 0, (size_t)units * sizeof(InstResult), st);
    SearchArgs SA = single_args(h, P, w, CSP_ALL, h->up_cap, lim);
    SA.batch = 1;
    SA.n_inst = (int32_t)units;
    SA.teams = (Team *)(w + P.o_team);
    SA.results = (InstResult *)(w + P.o_res);
    SA.roots = (const uint32_t *)A;
    SA.global_limits = 1;
    SA.part = 0;
    SA.nparts = 1;
    if (e == cudaSuccess && units > 0) e = launch_init_batch(SA, P.shape.blocks, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev2, st);
    if (e == cudaSuccess && units > 0)
        e = launch_search(W, P.shape.stage_words > 0, P.shape.kind, SA, P.shape.blocks,
                          P.shape.warps * 32, P.shape.smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, st);
    return e;
}

int csp_launch(csp_t *h, const csp_limits *lim) {
    if (!h || !h->uploaded) return CSP_ESTATE;
    const Plan &P = h->plan;
    if (P.split) {
        const cudaError_t e = split_launch(h, lim);
        h->stats.workers = P.shape.blocks * P.shape.warps;
        h->stats.blocks = P.shape.blocks;
        return cuda_status(e);
    }
    SearchArgs A = single_args(h, P, h->ws, h->up_mode, h->up_cap, lim);
    cudaError_t e = cudaMemsetAsync(h->ws + P.o_g, 0, sizeof(GState), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + P.o_team, 0, sizeof(Team), h->stream);
    if (e == cudaSuccess) e = launch_init_single(A, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev0, h->stream);
    if (e == cudaSuccess)
        e = launch_search(P.W, P.shape.stage_words > 0, P.shape.kind, A, P.shape.blocks,
                          P.shape.warps * 32, P.shape.smem, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, h->stream);
    h->stats.workers = P.shape.blocks * P.shape.warps;
    h->stats.blocks = P.shape.blocks;
    return cuda_status(e);
}

int csp_collect(csp_t *h, int32_t *sol_out) {
    if (!h || !h->uploaded || !h->pin_g) return CSP_ESTATE;
    const Plan &P = h->plan;
    cudaError_t e = cudaMemcpyAsync(h->pin_g, h->ws + P.o_g, sizeof(GState),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    GState g = *h->pin_g;
    if (P.split) {                      // the levels the split expanded
        g.nodes += h->split_nodes;
        g.fails += h->split_fails;
    }
    int64_t d2h = sizeof(GState);
    const int64_t cap = h->up_mode == CSP_FIRST ? 1 : h->up_cap;
    int64_t stored = std::min<int64_t>((int64_t)g.solutions, cap);
    if (h->up_mode == CSP_ALL) stored = std::min<int64_t>((int64_t)g.stored, cap);
    if (sol_out && stored > 0) {
        e = cudaMemcpyAsync(sol_out, h->ws + P.o_sols, (size_t)stored * h->n * 4,
                            cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        d2h += stored * h->n * 4;
    }
    float ms = 0.f, kms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (P.split) cudaEventElapsedTime(&kms, h->ev2, h->ev1);
    else kms = ms;
    cudaGetLastError();
    fill_stats(&h->stats, g, stored);
    h->stats.ms = ms;
    h->stats.kernel_ms = kms;
    h->stats.units = P.split ? h->split_units : 1;
    h->stats.status = g.status;
    h->stats.d2h_bytes = d2h;
    return g.status;
}

int csp_solve(csp_t *h, int32_t mode, int64_t cap, int32_t *sol_out, const csp_limits *lim) {
    if (!h) return CSP_EINVAL;
    if (cap > 0 && !sol_out) return CSP_EINVAL;
    int rc = csp_upload(h, mode, cap);
    if (rc) return rc;
    rc = csp_launch(h, lim);
    if (rc) return rc;
    return csp_collect(h, sol_out);
}

int csp_propagate(csp_t *h, int32_t count, const uint32_t *dom_in, uint32_t *dom_out,
                  int32_t *failed) {
    if (!h || count < 0 || (count > 0 && (!dom_in || !dom_out || !failed))) return CSP_EINVAL;
    if (h->tiling.threads_per_node == 16) return CSP_EINVAL;     // two nodes per warp: search only
    if (!h->ws) return CSP_ESTATE;
    if (count == 0) return CSP_OK;
    Plan L;
    std::vector<uint32_t> B;
    int rc = plan_single(h, CSP_PROPAGATE, count, &L, &B);
    if (rc) return rc;
    if (L.bytes > h->ws_bytes) return CSP_ENOMEM;
    h->uploaded = false;          // the workspace is overwritten
    const size_t sw = (size_t)h->n * h->W * 4;
    cudaError_t e = cudaMemcpyAsync(h->ws + L.o_inst, B.data(), B.size() * 4,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws + L.o_qseq, dom_in, sw * count, cudaMemcpyHostToDevice, h->stream);
    PropArgs P{};
    P.inst = (const uint32_t *)(h->ws + L.o_inst);
    P.din = (const uint32_t *)(h->ws + L.o_qseq);
    P.dout = (uint32_t *)(h->ws + L.o_qrec);
    P.failed = (int32_t *)(h->ws + L.o_sols);
    P.count = count;
    const int cons4 = ((int)B[H_CONS_WORDS] + 3) & ~3;
    const size_t per_state = (size_t)(((h->n * h->W + 3) & ~3) + 64) * 4;   // state, chg, evs
    const int tpn = h->tiling.threads_per_node;
    const bool block_per_node = tpn > 32;
    // a warp per state: up to 8 states per block, as many as fit; a block per state: tpn threads
    int warps = block_per_node ? tpn / 32 : 8;
    if (!block_per_node)
        while (warps > 1 && per_state * warps > SMEM_MAX) --warps;
    size_t smem = per_state * (block_per_node ? 1 : warps);
    P.stage_words = (smem + (size_t)cons4 * 4 <= SMEM_MAX) ? cons4 : 0;
    smem += (size_t)P.stage_words * 4;
    if (smem > SMEM_MAX) return CSP_ETOOBIG;
    const int per_block = block_per_node ? 1 : warps;
    const int blocks = std::max(1, std::min(4096, (count + per_block - 1) / per_block));
    if (e == cudaSuccess) e = cudaEventRecord(h->ev0, h->stream);
    if (e == cudaSuccess)
        e = launch_propagate(h->W, P.stage_words > 0, P, blocks, warps * 32, smem, h->stream,
                             block_per_node);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev1, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dom_out, h->ws + L.o_qrec, sw * count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(failed, h->ws + L.o_sols, 4 * (size_t)count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    // statistics of the call: one node per state, the failed ones, the kernel's device time
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    cudaGetLastError();
    int64_t nf = 0;
    for (int32_t k = 0; k < count; ++k) nf += failed[k] != 0;
    h->stats = csp_stats_t{};
    h->stats.nodes = (uint64_t)count;
    h->stats.fails = (uint64_t)nf;
    h->stats.ms = ms;
    h->stats.kernel_ms = ms;
    h->stats.blocks = blocks;
    h->stats.workers = block_per_node ? blocks : blocks * warps;
    h->stats.h2d_bytes = (int64_t)B.size() * 4 + (int64_t)sw * count;
    h->stats.d2h_bytes = (int64_t)(sw + 4) * count;
    return CSP_OK;
}

int csp_stats(const csp_t *h, csp_stats_t *out) {
    if (!h || !out) return CSP_EINVAL;
    *out = h->stats;
    return CSP_OK;
}

void csp_destroy(csp_t *h) {
    if (!h) return;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->pin_block) cudaFreeHost(h->pin_block);
    if (h->pin_g) cudaFreeHost(h->pin_g);
    cudaGetLastError();
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------- batches

// Layout of a batch workspace (as Plan for one problem).
struct BatchPlan {
    Shape shape;
    int R = 4;
    int depth = 2;                   // stack levels per worker
    int pairs = 0;                   // pairs possible (used in all-solution launches)
    size_t o_arena = 0, o_ioff = 0, o_soff = 0, o_g = 0, o_teams = 0, o_qseq = 0, o_qrec = 0,
           o_spill = 0, o_sols = 0, o_res = 0, o_mlp_params = 0, o_mlp_packed = 0;
    size_t bytes = 0;
};

struct csp_batch {
    std::vector<csp *> hs;
    int W = 1, depth = 2, cons_max = 0;
    std::vector<uint32_t> arena;
    std::vector<int64_t> inst_off, sol_off;
    int64_t pending_h2d = 0;         // bytes uploaded since the last collect
    int64_t sol_words = 0;
    csp_tiling tiling{0, 0, 0, 0};
    BatchPlan plan;                  // workspace layout of the last upload
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool uploaded = false;
    int32_t mode = -1;
    int nmax = 1, ntab_max = 0;
    bool all_reg = true;             // every instance has FLAG_NE_REG
    int32_t brancher = CSP_BR_FIRST_FAIL;
    std::vector<uint16_t> mlp_params;
    float *logbuf = nullptr;                 // subtree logging (caller-owned device buffers)
    unsigned long long *log_count = nullptr;
    int64_t log_cap = 0;
    uint32_t log_sample = 1;
    cudaGraphExec_t graph = nullptr;
    int32_t graph_mode = -1;
    csp_limits graph_lim{};
    csp_stats_t stats{};
};

namespace {

// Layout of the batch's workspace under its current tiling, brancher and logging; the
// batch is not modified.
int plan_batch(const csp_batch *b, BatchPlan *P) {
    BatchPlan p;
    const bool learned = b->brancher == CSP_BR_LEARNED;
    p.R = record_words(b->nmax * b->W, b->W, b->logbuf ? LOG_EXTRA : 0);
    // the plan does not know the mode: room for pairs wherever an all-solution launch may use them
    const int pairs = pairs_of(b->tiling, b->all_reg && !learned && !b->logbuf, b->nmax, true);
    if (pairs < 0) return pairs;
    p.pairs = pairs;
    p.depth = stack_depth(b->nmax, pairs > 0);
    int rc = make_shape(b->tiling, b->W, p.R, p.depth, b->cons_max, true, learned,
                        b->logbuf != nullptr, b->nmax, b->ntab_max, b->all_reg, &p.shape);
    if (rc) return rc;
    const Shape &s = p.shape;
    const size_t count = b->hs.size();
    Carver c;
    p.o_arena = c.take(b->arena.size() * 4);
    p.o_ioff = c.take(count * 8);
    p.o_soff = c.take(count * 8);
    p.o_g = c.take(sizeof(GState));
    p.o_teams = c.take((size_t)s.blocks * sizeof(Team));
    p.o_qseq = c.take((size_t)s.blocks * s.qcap * 4);
    p.o_qrec = c.take((size_t)s.blocks * s.qcap * p.R * 4);
    p.o_spill = c.take((size_t)s.blocks * s.warps * p.depth * p.R * 4);
    p.o_sols = c.take((size_t)std::max<int64_t>(b->sol_words, 1) * 4);
    p.o_res = c.take(count * sizeof(InstResult));
    p.o_mlp_params = c.take(learned ? CSP_MLP_PARAMS * 2 : 0);
    p.o_mlp_packed = c.take(learned ? CSP_MLP_PACKED_WORDS * 4 : 0);
    p.bytes = c.off;
    *P = p;
    return CSP_OK;
}

SearchArgs batch_args(csp_batch *b, const csp_limits *lim) {
    SearchArgs A{};
    uint8_t *w = b->ws;
    A.arena = (const uint32_t *)(w + b->plan.o_arena);
    A.inst_off = (const int64_t *)(w + b->plan.o_ioff);
    A.sol_off = (const int64_t *)(w + b->plan.o_soff);
    A.n_inst = (int32_t)b->hs.size();
    A.mode = b->mode;
    A.batch = 1;
    A.lsm = b->plan.shape.lsm;
    A.rmax = b->plan.R;
    A.depth = b->plan.depth;
    A.pairs = b->plan.pairs && b->mode == CSP_ALL;
    A.stage_words = b->plan.shape.stage_words;
    A.qmask = b->plan.shape.qcap - 1;
    A.flags = lim ? lim->flags : 0;
    A.warps = b->plan.shape.warps;
    A.g = (GState *)(w + b->plan.o_g);
    A.teams = (Team *)(w + b->plan.o_teams);
    A.qseq = (uint32_t *)(w + b->plan.o_qseq);
    A.qrec = (uint32_t *)(w + b->plan.o_qrec);
    A.spill = (uint32_t *)(w + b->plan.o_spill);
    A.sols = (int32_t *)(w + b->plan.o_sols);
    A.cap = 0;
    A.results = (InstResult *)(w + b->plan.o_res);
    A.node_limit = lim ? lim->node_limit : 0;
    A.deadline_ns = lim ? lim->time_limit_ns : 0;
    A.wait_limit_ns = (lim && lim->wait_limit_ns > 0) ? lim->wait_limit_ns : 60000000000LL;
    set_learned_args(A, b->plan.shape, b->brancher == CSP_BR_LEARNED, w, b->plan.o_mlp_packed);
    A.log_extra = b->logbuf ? LOG_EXTRA : 0;
    A.log_sample = b->log_sample;
    A.logbuf = b->logbuf;
    A.log_count = b->log_count;
    A.log_cap = b->log_cap;
    if (b->logbuf) A.flags |= CSP_F_NO_DONATE;      // a level's subtree must stay with one worker
    A.part = 0;
    A.nparts = 1;
    return A;
}

cudaError_t enqueue_batch(csp_batch *b, const SearchArgs &A) {
    cudaError_t e = cudaMemsetAsync(b->ws + b->plan.o_g, 0, sizeof(GState), b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->ws + b->plan.o_teams, 0, (size_t)b->plan.shape.blocks * sizeof(Team), b->stream);
    if (e == cudaSuccess)   // per-instance counters are accumulated atomically by every helper
        e = cudaMemsetAsync(b->ws + b->plan.o_res, 0, b->hs.size() * sizeof(InstResult), b->stream);
    if (e == cudaSuccess) e = launch_init_batch(A, b->plan.shape.blocks, b->stream);
    if (e == cudaSuccess)
        e = launch_search(b->W, b->plan.shape.stage_words > 0, b->plan.shape.kind, A, b->plan.shape.blocks,
                          b->plan.shape.warps * 32, b->plan.shape.smem, b->stream);
    return e;
}

void drop_graph(csp_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_mode = -1;
}

bool same_limits(const csp_limits &a, const csp_limits &b) {
    return a.node_limit == b.node_limit && a.time_limit_ns == b.time_limit_ns &&
           a.wait_limit_ns == b.wait_limit_ns && a.flags == b.flags;
}

}  // namespace

extern "C" {

int csp_batch_create(csp_batch_t **out, csp_t *const *hs, int32_t count) {
    if (!out || count < 1 || !hs) return CSP_EINVAL;
    for (int i = 0; i < count; ++i) if (!hs[i]) return CSP_EINVAL;
    csp_batch *b = new csp_batch();
    b->hs.assign(hs, hs + count);
    int W = 1, nmax = 1;
    for (csp *h : b->hs) { W = std::max(W, h->W); nmax = std::max(nmax, h->n); }
    b->W = W;
    b->nmax = nmax;
    b->depth = nmax + 1;
    int64_t sw = 0;
    for (csp *h : b->hs) {
        std::vector<uint32_t> B;
        encode(h, W, B);
        b->inst_off.push_back((int64_t)b->arena.size());
        b->arena.insert(b->arena.end(), B.begin(), B.end());
        b->cons_max = std::max(b->cons_max, (int)B[H_CONS_WORDS]);
        b->ntab_max = std::max(b->ntab_max, (int)B[H_N_TAB]);
        b->all_reg = b->all_reg && (B[H_FLAGS] & FLAG_NE_REG) != 0;
        b->sol_off.push_back(sw);
        sw += h->n;
    }
    b->sol_words = sw;
    *out = b;
    return CSP_OK;
}

int csp_batch_create_roots(csp_batch_t **out, csp_t *base, int32_t count, const uint32_t *roots) {
    if (!out || !base || count < 1 || !roots) return CSP_EINVAL;
    csp_batch *b = new csp_batch();
    b->hs.assign((size_t)count, base);
    const int W = base->W, n = base->n;
    b->W = W;
    b->nmax = n;
    b->depth = n + 1;
    std::vector<uint32_t> B;
    encode(base, W, B);
    const size_t root = B[H_OFF_ROOT], S = (size_t)n * W;
    b->arena.resize(B.size() * (size_t)count);
    for (int i = 0; i < count; ++i) {
        const size_t off = B.size() * (size_t)i;
        std::memcpy(&b->arena[off], B.data(), B.size() * 4);
        for (size_t k = 0; k < S; ++k) b->arena[off + root + k] = B[root + k] & roots[S * i + k];
        b->inst_off.push_back((int64_t)off);
        b->sol_off.push_back((int64_t)n * i);
    }
    b->cons_max = (int)B[H_CONS_WORDS];
    b->ntab_max = (int)B[H_N_TAB];
    b->all_reg = (B[H_FLAGS] & FLAG_NE_REG) != 0;
    b->sol_words = (int64_t)n * count;
    *out = b;
    return CSP_OK;
}

int csp_batch_set_tiling(csp_batch_t *b, const csp_tiling *t) {
    if (!b) return CSP_EINVAL;
    csp_tiling nt = t ? *t : csp_tiling{0, 0, 0, 0, 0, 0, 0};
    if (!tiling_ok(nt)) return CSP_EINVAL;
    if (nt.domain_words != 0 && nt.domain_words != b->W) return CSP_EINVAL;   // arena encoded at b->W
    b->tiling = nt;
    b->uploaded = false;
    drop_graph(b);
    return CSP_OK;
}

int csp_batch_workspace_bytes(const csp_batch_t *bc, int32_t mode, size_t *bytes) {
    if (!bc || !bytes || mode < 0 || mode > 1) return CSP_EINVAL;
    BatchPlan P;
    const int rc = plan_batch(bc, &P);
    if (rc) return rc;
    *bytes = P.bytes;
    return CSP_OK;
}

int csp_batch_set_brancher(csp_batch_t *b, int32_t kind, const uint16_t *bf16_weights) {
    if (!b || (kind != CSP_BR_FIRST_FAIL && kind != CSP_BR_LEARNED)) return CSP_EINVAL;
    if (kind == CSP_BR_LEARNED) {
        if (bf16_weights) b->mlp_params.assign(bf16_weights, bf16_weights + CSP_MLP_PARAMS);
        if (b->mlp_params.size() != (size_t)CSP_MLP_PARAMS) return CSP_EINVAL;
    }
    b->brancher = kind;
    b->uploaded = false;
    drop_graph(b);
    return CSP_OK;
}

int csp_batch_set_log(csp_batch_t *b, float *log_dev, unsigned long long *count_dev, int64_t cap,
                      uint32_t sample) {
    if (!b || cap < 0 || (cap > 0 && (!log_dev || !count_dev))) return CSP_EINVAL;
    b->logbuf = cap > 0 ? log_dev : nullptr;
    b->log_count = cap > 0 ? count_dev : nullptr;
    b->log_cap = cap;
    b->log_sample = sample < 1 ? 1 : sample;
    b->uploaded = false;
    drop_graph(b);
    return CSP_OK;
}

int csp_batch_bind(csp_batch_t *b, void *dev, size_t bytes, void *cuda_stream) {
    if (!b || !dev || ((uintptr_t)dev % ALIGN)) return CSP_EINVAL;
    if (!b->ev0) {
        if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
            cudaGetLastError();
            return CSP_ECUDA;
        }
    }
    b->ws = (uint8_t *)dev;
    b->ws_bytes = bytes;
    b->stream = (cudaStream_t)cuda_stream;
    b->uploaded = false;
    drop_graph(b);
    return CSP_OK;
}

static int batch_upload(csp_batch *b, int32_t mode) {
    if (!b->ws) return CSP_ESTATE;
    BatchPlan P;
    int rc = plan_batch(b, &P);
    if (rc) return rc;
    if (P.bytes > b->ws_bytes) return CSP_ENOMEM;
    // from here on the workspace is overwritten: the previous upload (and any graph that
    // launches it) is no longer valid
    b->uploaded = false;
    drop_graph(b);
    b->plan = P;
    const size_t count = b->hs.size();
    cudaError_t e = cudaMemcpyAsync(b->ws + P.o_arena, b->arena.data(), b->arena.size() * 4,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ws + P.o_ioff, b->inst_off.data(), count * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ws + P.o_soff, b->sol_off.data(), count * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->brancher == CSP_BR_LEARNED)
        e = upload_mlp(b->mlp_params, b->ws, P.o_mlp_params, P.o_mlp_packed, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    b->mode = mode;
    b->uploaded = true;
    b->pending_h2d += (int64_t)b->arena.size() * 4 + (int64_t)count * 16 +
                      (b->brancher == CSP_BR_LEARNED ? (int64_t)CSP_MLP_PARAMS * 2 : 0);
    return CSP_OK;
}

int csp_batch_launch(csp_batch_t *b, const csp_limits *lim, int32_t use_graph) {
    if (!b || !b->uploaded) return CSP_ESTATE;
    if (b->tiling.threads_per_node == 16 && b->mode != CSP_ALL) return CSP_EINVAL;
    const csp_limits L = lim ? *lim : csp_limits{0, 0, 0, 0, 0};
    SearchArgs A = batch_args(b, &L);
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        if (!b->stream) return CSP_EINVAL;      // the legacy stream cannot be captured
        if (!b->graph || b->graph_mode != b->mode || !same_limits(L, b->graph_lim)) {
            drop_graph(b);
            int bps = 0;   // sets the kernel's shared-memory attribute outside the capture
            e = occupancy_search(b->W, b->plan.shape.stage_words > 0, b->plan.shape.kind, b->plan.shape.warps * 32,
                                 b->plan.shape.smem, &bps);
            cudaGraph_t g = nullptr;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                cudaError_t e1 = enqueue_batch(b, A);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) { drop_graph(b); return cuda_status(e); }
            b->graph_mode = b->mode;
            b->graph_lim = L;
        }
        e = cudaEventRecord(b->ev0, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
    } else {
        e = cudaEventRecord(b->ev0, b->stream);
        if (e == cudaSuccess) e = enqueue_batch(b, A);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->stream);
    b->stats.workers = b->plan.shape.blocks * b->plan.shape.warps;
    b->stats.blocks = b->plan.shape.blocks;
    return cuda_status(e);
}

int csp_batch_collect(csp_batch_t *b, csp_result *out, int32_t *sol) {
    if (!b || !b->uploaded) return CSP_ESTATE;
    const size_t count = b->hs.size();
    GState g;
    std::vector<InstResult> res(count);
    cudaError_t e = cudaMemcpyAsync(&g, b->ws + b->plan.o_g, sizeof(g), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), b->ws + b->plan.o_res, count * sizeof(InstResult),
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && sol)
        e = cudaMemcpyAsync(sol, b->ws + b->plan.o_sols, (size_t)b->sol_words * 4, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (out)
        for (size_t i = 0; i < count; ++i) {
            out[i].status = res[i].status;
            out[i].n = b->hs[i]->n;
            out[i].nodes = res[i].nodes;
            out[i].fails = res[i].fails;
            out[i].solutions = res[i].solutions;
            out[i].sol_offset = b->sol_off[i];
            out[i].ms = res[i].t_end > res[i].t_start ? 1e-6 * (double)(res[i].t_end - res[i].t_start) : 0.0;
        }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    cudaGetLastError();
    fill_stats(&b->stats, g, 0);
    b->stats.ms = ms;
    b->stats.kernel_ms = ms;
    b->stats.units = (int64_t)b->hs.size();
    b->stats.status = g.status;
    b->stats.h2d_bytes = b->pending_h2d;
    b->pending_h2d = 0;
    b->stats.d2h_bytes = (int64_t)sizeof(g) + (int64_t)(count * sizeof(InstResult)) +
                         (sol ? b->sol_words * 4 : 0);
    return g.status;
}

int csp_batch_solve(csp_batch_t *b, int32_t mode, const csp_limits *lim, int32_t use_graph,
                    csp_result *out, int32_t *sol) {
    if (!b || mode < 0 || mode > 1) return CSP_EINVAL;
    if (!b->uploaded || b->mode != mode) {
        int rc = batch_upload(b, mode);
        if (rc) return rc;
    }
    int rc = csp_batch_launch(b, lim, use_graph);
    if (rc) return rc;
    return csp_batch_collect(b, out, sol);
}

int64_t csp_batch_solution_words(const csp_batch_t *b) { return b ? b->sol_words : 0; }

int csp_batch_stats(const csp_batch_t *b, csp_stats_t *out) {
    if (!b || !out) return CSP_EINVAL;
    *out = b->stats;
    return CSP_OK;
}

void csp_batch_destroy(csp_batch_t *b) {
    if (!b) return;
    drop_graph(b);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    cudaGetLastError();
    delete b;
}

int csp_probe_smem_bandwidth(void *dev_out, void *cuda_stream, int32_t reps, double *gbs) {
    if (!dev_out || !gbs || reps < 1) return CSP_EINVAL;
    DeviceInfo di = device_info();
    if (!di.ok) return CSP_ECUDA;
    return cuda_status(probe_smem(dev_out, (cudaStream_t)cuda_stream, di.sms, reps, gbs));
}

}  // extern "C"

// ---------------------------------------------------------------------------- no-alloc search

namespace {

// Scratch of csp_solve_noalloc, part of the library's device image: every GPU that loads
// the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CSP_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES];   // device address of the array, per device

}  // namespace

extern "C" {

int csp_solve_noalloc(csp_t *h, int32_t mode, int64_t cap, int32_t *sol_out,
                      const csp_limits *lim, void *cuda_stream) {
    if (!h || mode < 0 || mode > 1 || cap < 0 || cap > INT32_MAX) return CSP_EINVAL;
    if (cap > 0 && !sol_out) return CSP_EINVAL;
    // The call waits for the device and copies from pageable host memory, neither of which
    // may happen on a capturing stream (it would invalidate the caller's capture): refused
    // before anything else is done.
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            return CSP_ECUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return CSP_ESTATE;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CSP_ECUDA; }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return CSP_ECUDA;
    // Lay the search out in the array as it would be in a bound workspace.  The plan is
    // local: the handle's own binding, upload and plan are left as they were, so a workspace
    // bound and uploaded earlier can still be launched after this call, whatever it returns.
    Plan P;
    std::vector<uint32_t> B;
    int rc = plan_single(h, mode, cap, &P, &B, false);
    if (rc) return rc;
    if (P.bytes > (size_t)CSP_NOALLOC_SCRATCH_BYTES) return CSP_ENOMEM;
    if (!g_noalloc_ptr[dev]) {
        // set-up, once per device with that device current: the host-side name of the
        // array is not a device address, so look the address up
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CSP_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    uint8_t *const ws = (uint8_t *)g_noalloc_ptr[dev];
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool learned = h->brancher == CSP_BR_LEARNED;
    const int64_t zero = 0;
    SearchArgs A = single_args(h, P, ws, mode, cap, lim);
    cudaError_t e = cudaMemcpyAsync(ws + P.o_inst, B.data(), B.size() * 4,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + P.o_off, &zero, sizeof(zero), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && learned)
        e = upload_mlp(h->mlp_params, ws, P.o_mlp_params, P.o_mlp_packed, st);
    // the launch counters and the work queue's state start at zero on every call
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + P.o_g, 0, sizeof(GState), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + P.o_team, 0, sizeof(Team), st);
    if (e == cudaSuccess) e = launch_init_single(A, st);
    if (e == cudaSuccess)
        e = launch_search(P.W, P.shape.stage_words > 0, P.shape.kind, A, P.shape.blocks,
                          P.shape.warps * 32, P.shape.smem, st);
    GState g;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g, ws + P.o_g, sizeof(g), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int64_t stored = 0;
    if (e == cudaSuccess) {
        const int64_t c1 = mode == CSP_FIRST ? 1 : cap;
        stored = std::min<int64_t>(mode == CSP_ALL ? (int64_t)g.stored : (int64_t)g.solutions, c1);
        if (sol_out && stored > 0) {
            e = cudaMemcpyAsync(sol_out, ws + P.o_sols, (size_t)stored * h->n * 4,
                                cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    if (e != cudaSuccess) return cuda_status(e);
    fill_stats(&h->stats, g, stored);
    h->stats.ms = 0.0;
    h->stats.kernel_ms = 0.0;
    h->stats.units = 1;
    h->stats.status = g.status;
    h->stats.workers = P.shape.blocks * P.shape.warps;
    h->stats.blocks = P.shape.blocks;
    h->stats.h2d_bytes = (int64_t)B.size() * 4 + (int64_t)sizeof(int64_t) +
                         (learned ? (int64_t)CSP_MLP_PARAMS * 2 : 0);
    h->stats.d2h_bytes = (int64_t)sizeof(GState) + stored * h->n * 4;
    return g.status;
}

const char *csp_strerror(int code) {
    switch (code) {
    case CSP_OK: return "ok";
    case CSP_EINVAL: return "invalid argument";
    case CSP_ENOMEM: return "workspace too small";
    case CSP_ETOOBIG: return "problem exceeds supported sizes";
    case CSP_ECUDA: return "CUDA error or no device";
    case CSP_ELIMIT: return "node or time limit reached";
    case CSP_ETIMEOUT: return "device-side wait limit exceeded";
    case CSP_ESTATE: return "call out of order";
    default: return "unknown error";
    }
}

}  // extern "C"
