// CUBICS search kernels for sm_103a (arxiv 1909.09213, Sections 2.1-2.3).
//
// The whole search stays on the GPU (Section 2.1).  One warp is one worker: it owns a
// depth-first stack of search levels, labels one variable per level (d-way, values
// ascending), propagates each child to its fixpoint and backtracks on failure.  Each level
// is a full copy of the parent's domains plus the values still to try, so backtracking is
// a restore of one record: the copy is parallel over the domain words (the per-domain
// save/restore of Section 2.2), done by the 32 lanes.  The top levels of each stack live
// in shared memory (Section 2.3); deeper ones spill to a private global-memory area.
//
// Idle workers take records (a parent state with untried values) from a work queue; busy
// workers donate their shallowest untried values when someone is idle (search-space
// partitioning with a task pool, Section 1.3).  In single-problem mode the team is the whole
// grid; in batch mode each block is a team that solves one instance after another.
//
// Included by one translation unit per domain width W (kernels_w*.cu).
#pragma once
#include <cuda_runtime.h>
#include "device.cuh"
#include "mlp.cuh"

namespace cubics {

constexpr int CSP_EINVAL_ = -1;
constexpr int CSP_ELIMIT_ = -5;
constexpr int CSP_ETIMEOUT_ = -6;
constexpr int F_NO_DONATE = 1;

// launch arguments, copied once per block into shared memory
static __shared__ SearchArgs SA;

// per-warp bookkeeping kept in shared memory (lane 0 writes the counters)
struct WarpShared {
    uint32_t chg[32], evs[32];
    unsigned long long nodes, fails, sols, hsum, hxor, evals, steals, spills;
    long long t_start;
    int64_t sol_off;
    long long wait_ns;    // time spent waiting for a record
    int32_t maxd;
    int32_t hcnt;         // register kernel: solutions waiting in the hash buffer
    unsigned long long rounds;   // fixpoint rounds
    int32_t pad2[2];
};
static_assert(sizeof(WarpShared) == 4 * WS_WORDS, "WarpShared size must match WS_WORDS");

// ------------------------------------------------------------------ work queue
// Bounded ring of records with a sequence word per slot.  Producers claim a position with
// a compare-and-swap on the tail (a full queue makes the push fail, and the donor keeps its
// values).  Consumers take a ticket with a fetch-and-add on the head, which never fails,
// and wait for their own slot to be filled: waiting workers poll distinct words instead of
// all racing for the head, and they are served in ticket order.  Donors count the records
// they will push in the team's `promised` (an atomic addition before the push), and give
// only while head - promised > 0, so that the busy workers, who all see the same waiting
// workers, do not all donate to them.  Slot p & qmask holds sequence p when free for the
// producer of position p, and p + 1 once it holds that position's record.

// Claims the tail position for a push; returns it, or -1 when the queue is full.
__device__ __forceinline__ long long q_claim_tail(uint32_t *tail, const uint32_t *seq,
                                                  uint32_t qmask) {
    uint32_t pos = ld_volatile(tail);
    for (int it = 0; it < 256; ++it) {
        const int dif = (int)(ld_acquire(&seq[pos & qmask]) - pos);
        if (dif == 0) {
            const uint32_t prev = atomicCAS(tail, pos, pos + 1);
            if (prev == pos) return (long long)pos;
            pos = prev;
        } else if (dif < 0) {
            return -1;                     // the consumer of the previous lap is still copying
        } else {
            pos = ld_volatile(tail);
        }
    }
    return -1;
}

// Push a record of R words.  The source is shared memory at `src_sm` (>= 0) or global
// memory at `src_g`; lanes < W may replace the untried-value words by `my_rem`.
static __device__ bool q_push(Team *T, uint32_t *seq, uint32_t *rec, int src_sm, const uint32_t *src_g,
                       int R, int S, int W, bool override_rem, uint32_t my_rem) {
    const int lane = lane_id();
    long long pos = -1;
    if (lane == 0) pos = q_claim_tail(&T->tail, seq, (uint32_t)SA.qmask);
    pos = __shfl_sync(FULLMASK, pos, 0);
    if (pos < 0) return false;
    uint32_t *dst = rec + (size_t)((uint32_t)pos & (uint32_t)SA.qmask) * SA.rmax;
    if (src_sm >= 0) copy_sg(dst, src_sm, R);
    else copy_gg(dst, src_g, R);
    __syncwarp();
    if (override_rem && lane < W) dst[S + lane] = my_rem;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(&seq[(uint32_t)pos & (uint32_t)SA.qmask], (uint32_t)pos + 1u);
    return true;
}

// Receive the record of consumer ticket `t` into shared memory at `dst`, if it is there.
static __device__ bool q_take(uint32_t *seq, uint32_t *rec, uint32_t t, int dst, int R) {
    const int lane = lane_id();
    const uint32_t slot = t & (uint32_t)SA.qmask;
    int ready = 0;
    if (lane == 0) ready = ld_acquire(&seq[slot]) == t + 1u;
    if (!__shfl_sync(FULLMASK, ready, 0)) return false;
    __threadfence();
    copy_gs_cg(dst, rec + (size_t)slot * SA.rmax, R);
    __syncwarp();
    __threadfence();
    if (lane == 0) st_release(&seq[slot], t + (uint32_t)SA.qmask + 1u);
    return true;
}

// longest back-off between two polls of an empty queue
#ifndef CUBICS_POLL_MAX_NS
#define CUBICS_POLL_MAX_NS 8192u
#endif

// nodes a worker explores in a record before it may donate from it
#ifndef CUBICS_DONATE_AFTER
#define CUBICS_DONATE_AFTER 0u
#endif

// Records whose subtrees took less time on average (ns) are not worth passing through the
// queue: the donor's push and the taker's copy cost more than they spread.  The whole grid
// sharing one queue (single problem) pays more per record than a block's queue (batch).
#ifndef CUBICS_SMALL_NS_GRID
#define CUBICS_SMALL_NS_GRID 80000.f
#endif
#ifndef CUBICS_SMALL_NS_BATCH
#define CUBICS_SMALL_NS_BATCH 30000.f
#endif
// The same for the register-held kernel's single-problem queue.  Its nodes are ~3x shorter,
// and every record passed costs ~10 global atomics on the few counters of the team, so that
// many small records make the whole grid wait on those addresses (measured with 4864
// workers: 16-queens 0.9 G nodes/s at 160 us, 3.3 G at 640 us, 3.2 G at 1.28 ms; 15-queens
// 0.6 G at 640 us, 1.7 G at 1.28 ms)
#ifndef CUBICS_SMALL_NS_GRID_REG
#define CUBICS_SMALL_NS_GRID_REG 1280000.f
#endif
#ifndef CUBICS_REG_THR_FLOOR
#define CUBICS_REG_THR_FLOOR 0.0625f
#endif
// 1: a size bin's statistics count only finished records (a record still running is no
// evidence that its bin is small, so the first levels of a search are passed on at once);
// 0: running records are credited the nodes explored so far
#ifndef CUBICS_FINISHED_STATS
#define CUBICS_FINISHED_STATS 1
#endif

// records observed in a bin before its statistics are trusted
#ifndef CUBICS_USTAT_MIN
#define CUBICS_USTAT_MIN 8u
#endif

// while workers wait for records, a busy worker checks the donation signal every this many
// nodes (every 8th node otherwise); a block's own queue (batch mode) every node: only the
// grid-wide queue's counters are contended enough to make frequent checks cost
#ifndef CUBICS_HUNGRY_EVERY
#define CUBICS_HUNGRY_EVERY 4u
#endif

// nodes between two reads of the stop flags by a worker whose nodes are held in registers
// (its nodes are short: a read per node would wait on a global load every node)
#ifndef CUBICS_POLL_EVERY
#define CUBICS_POLL_EVERY 16u
#endif

// most records one donation check may push
// the paired expansion (two sibling nodes per warp) inline in the search loop, or a call
#ifndef CUBICS_PAIR_INLINE
#define CUBICS_PAIR_INLINE __forceinline__
#endif
#ifndef CUBICS_DONATE_MAX
#define CUBICS_DONATE_MAX 16
#endif

// ------------------------------------------------------------------ worker

// EXT: the worker can run the learned brancher and subtree logging.  Without them the
// search compiles into a separate kernel that fits in fewer registers (more resident warps).
// REG: one-word int_ne problems with at most 32 variables (FLAG_NE_REG); a node's domains are
// propagated and labelled in registers, one variable per lane, and reach shared memory only
// when the node opens a search level (records keep the layout of the other kernels).
template <int W, bool ST, bool EXT, bool REG = false>
struct Worker {
    IV<ST> I;
    Team *T;
    int slots;            // SM offset of the lsm stack records
    int wso;              // SM offset of this warp's WarpShared
    int lsm, R, S;
    int top, base;        // open levels [0, top); levels >= base are in shared memory
    uint32_t tick;        // nodes of this worker (low bits pace the periodic checks)
    int hungry;           // the last donation check saw workers waiting for records
    uint32_t worth_bins;  // bit b: records of size bin b are worth passing on (refreshed with
                          // the limits, every 64 nodes, from the team's subtree statistics)
    int owed_seen;        // workers waiting for a record at the last donation check
    uint32_t taken;       // tick when the current record was taken
    int pbin;             // size-statistics bin of the current record
    uint32_t credited;    // tick up to which its nodes were added to the bin
    int gw;               // global worker index
    int team;             // batch: index of the team (its queue) being helped
    int inst;             // batch: instance being searched
    int stop;             // a poll saw the stop flag
    // register kernel: node statistics since they were last added to WarpShared, packed in
    // two words (nodes in the low half of cnt_nf, fails in the high half; propagator
    // evaluations and fixpoint rounds likewise in cnt_er); added every 64 ticks (at most 128
    // nodes), so no half overflows (a node evaluates each of its at most 32 variables once,
    // in at most 33 rounds)
    uint32_t cnt_nf, cnt_er;

    __device__ __forceinline__ WarpShared &ws() const {
        return *reinterpret_cast<WarpShared *>(&SM[wso]);
    }
    __device__ __forceinline__ int chg() const { return wso; }
    __device__ __forceinline__ int evs() const { return wso + 32; }
    __device__ __forceinline__ uint32_t *qseq() const {
        return SA.qseq + (SA.batch ? (size_t)team * (SA.qmask + 1) : 0);
    }
    __device__ __forceinline__ uint32_t *qrec() const {
        return SA.qrec + (SA.batch ? (size_t)team * (SA.qmask + 1) * SA.rmax : 0);
    }
    __device__ __forceinline__ uint32_t *spill(int k) const {
        return SA.spill + ((size_t)gw * SA.depth + k) * SA.rmax;
    }
    // lsm is a power of two
    __device__ __forceinline__ int slot(int k) const { return slots + (k & (lsm - 1)) * R; }

    // Whether this node checks for workers owed a record: every 8th node; every node (a
    // block's queue) or every CUBICS_HUNGRY_EVERY-th (the grid's) while workers are starved
    // (ramp-up and the tail); never in the first nodes of a record, so that small subtrees
    // are not passed on.  The launch's flags are read only once the register test passes.
    __device__ __forceinline__ bool donation_due() const {
        if (!hungry && (tick & 7u) != 0u) return false;
        return !(SA.flags & F_NO_DONATE) &&
               ((tick & (hungry ? (SA.batch ? 0u : CUBICS_HUNGRY_EVERY - 1u) : 7u)) == 0u) &&
               tick - taken >= CUBICS_DONATE_AFTER;
    }

    // add the packed node statistics to WarpShared (whole warp)
    __device__ __forceinline__ void fold_counts() {
        if (lane_id() == 0 && (cnt_nf | cnt_er)) {
            WarpShared &w = ws();
            w.nodes += cnt_nf & 0xffffu;
            w.fails += cnt_nf >> 16;
            w.evals += cnt_er & 0xffffu;
            w.rounds += cnt_er >> 16;
        }
        cnt_nf = cnt_er = 0u;
    }

    // make the shared slot of level k (== top) free
    __device__ void make_room(int k) {
        const int old = k - lsm;
        if (old >= base) {
            copy_sg(spill(old), slot(old), R);
            __syncwarp();
            base = old + 1;
            if (lane_id() == 0) ws().spills++;
        }
    }
    // after a pop: the new top level must be in shared memory
    __device__ void refill() {
        if (top > 0 && top - 1 < base) {
            const int k = top - 1;
            copy_gs_cg(slot(k), spill(k), R);
            __syncwarp();
            base = k;
        }
    }

    // Issue the loads of the stop flags now; their value is consumed after the next node.
    __device__ __forceinline__ int poll() const {
        int s = 0;
        if (lane_id() == 0) {
            s = ld_volatile(&SA.g->abort);
            if (SA.mode == 1 || SA.batch) s |= ld_volatile(&T->found);
        }
        return s;
    }

    // Node and time limits, every 64 nodes.  In batch mode the node limit is per instance:
    // the team's instance stops (found = 2) and the others go on.
    __device__ __noinline__ void check_limits() {
        // nodes since the last check: 64 ticks, or the register kernel's own count (a tick
        // of a pair is two nodes)
        unsigned long long nn = 64ull;
        if constexpr (REG) {
            nn = cnt_nf & 0xffffu;
            fold_counts();
        }
        refresh_worth();
        if (lane_id() == 0) {
            if (!CUBICS_FINISHED_STATS) {
                atomicAdd(&T->usum[pbin], (unsigned long long)(tick - credited));
                credited = tick;
            }
            if (SA.node_limit > 0 && SA.batch && !SA.global_limits) {
                const unsigned long long tot = atomicAdd(&T->progress, nn) + nn;
                if ((long long)tot >= SA.node_limit) atomicCAS(&T->found, 0, 2);
            } else if (SA.node_limit > 0) {
                const unsigned long long tot = atomicAdd(&SA.g->node_progress, nn) + nn;
                if ((long long)tot >= SA.node_limit) {
                    atomicCAS(&SA.g->status, 0, CSP_ELIMIT_);
                    atomicExch(&SA.g->abort, 1);
                }
            }
            if (SA.deadline_ns > 0 && global_ns() - ws().t_start > SA.deadline_ns) {
                atomicCAS(&SA.g->status, 0, CSP_ELIMIT_);
                atomicExch(&SA.g->abort, 1);
            }
        }
    }

    // Which size bins are worth donating: a bin's records took, on average, its mean nodes
    // times the team's mean time per node; bins with too few records observed count as
    // worth it.  One lane per bin.
    __device__ void refresh_worth() {
        const int lane = lane_id();
        const uint32_t cnt = ld_volatile(&T->ucnt[lane]);
        const unsigned long long sum = ld_volatile(&T->usum[lane]);
        const unsigned long long xn = ld_volatile(&T->xnodes);
        const unsigned long long xs = ld_volatile(&T->xns);
        bool w = true;
        if (cnt >= CUBICS_USTAT_MIN && xn > 0) {
            const float mean_nodes = (float)sum / (float)cnt;
            const float node_ns = (float)xs / (float)xn;
            float thr = SA.batch ? CUBICS_SMALL_NS_BATCH
                                 : (REG ? CUBICS_SMALL_NS_GRID_REG : CUBICS_SMALL_NS_GRID);
            if (REG && !SA.batch) {
                // the more workers wait, the smaller the records worth passing on: a waiting
                // worker's time is lost anyway (down to CUBICS_REG_THR_FLOOR of the threshold)
                const float busy = 1.f - (float)owed_seen / (float)(gridDim.x * SA.warps);
                thr *= fmaxf(busy, CUBICS_REG_THR_FLOOR);
            }
            w = mean_nodes * node_ns >= thr;
        }
        worth_bins = __ballot_sync(FULLMASK, w);
    }

    __device__ void record_solution(int st) {
        const int lane = lane_id();
        const int n = I.n;
        bool keep = true;
        if (SA.mode == 1) {
            int won = 0;
            if (lane == 0) won = atomicCAS(&T->found, 0, 1) == 0;
            keep = __shfl_sync(FULLMASK, won, 0) != 0;
            stop = 1;         // this worker saw a solution: no further node in FIRST mode
        }
        if (!keep) return;
        if (lane == 0) {
            unsigned long long h = 0x9E3779B97F4A7C15ull;
            for (int i = 0; i < n; ++i) {
                const unsigned val = (unsigned)(I.lo0 + dom_min<W>(st + i * W));
                h = splitmix64(h ^ (((unsigned long long)(unsigned)i << 32) | val));
            }
            WarpShared &w = ws();
            w.sols++;
            w.hsum += h;
            w.hxor ^= h;
            if (SA.batch) atomicAdd(&SA.results[inst].solutions, 1ull);
        }
        long long slot_off = -1;
        if (SA.mode == 1) {
            slot_off = ws().sol_off;
        } else if (SA.cap > 0) {
            unsigned long long s = 0;
            if (lane == 0 && ld_volatile((const uint32_t *)&SA.g->stored) < (uint32_t)SA.cap)
                s = atomicAdd(&SA.g->stored, 1ull) + 1ull;
            s = __shfl_sync(FULLMASK, s, 0);
            if (s > 0 && (long long)s <= SA.cap) slot_off = (long long)(s - 1) * n;
        }
        if (slot_off >= 0 && SA.sols != nullptr)
            for (int i = lane; i < n; i += 32) SA.sols[slot_off + i] = I.lo0 + dom_min<W>(st + i * W);
        __syncwarp();
    }

    // SM offset of the warp's deferred solution-hash buffer (register kernel)
    __device__ __forceinline__ int hbuf() const {
        return wso + WS_WORDS + SA.feat_words + SA.list_words;
    }

    // Hash the solutions waiting in the buffer, one per lane (each lane runs one solution's
    // chain of n splitmix64 steps, the same chain as record_solution), and add their sum and
    // xor to WarpShared.  Whole warp.
    __device__ __noinline__ void hash_flush_reg() {
        const int lane = lane_id();
        const int n = I.n;
        WarpShared &w = ws();
        const int waiting = w.hcnt;
        unsigned long long h = 0ull, hx = 0ull;
        if (lane < waiting) {
            const uint32_t *row = &SM[hbuf() + lane * HB_STRIDE];
            h = 0x9E3779B97F4A7C15ull;
            uint32_t word = 0u;
            for (int i = 0; i < n; ++i) {
                if ((i & 3) == 0) word = row[i >> 2];
                const unsigned vi = (unsigned)(I.lo0 + (int)((word >> ((i & 3) * 8)) & 0xffu));
                h = splitmix64(h ^ (((unsigned long long)(unsigned)i << 32) | vi));
            }
            hx = h;
        }
        for (int o = 16; o > 0; o >>= 1) {
            h += __shfl_xor_sync(FULLMASK, h, o);
            hx ^= __shfl_xor_sync(FULLMASK, hx, o);
        }
        __syncwarp();
        if (lane == 0) {
            w.hsum += h;
            w.hxor ^= hx;
            w.hcnt = 0;
        }
        __syncwarp();
    }

    // record_solution for a node held in registers (lane i: the one value of x_i).  The
    // solution hash is deferred: the values (offsets from lo0, one byte each) go to the
    // warp's buffer, and every HB_SOLS solutions hash_flush_reg hashes them together.
    __device__ __noinline__ void record_solution_reg(uint32_t d) {
        const int lane = lane_id();
        const int n = I.n;
        bool keep = true;
        if (SA.mode == 1) {
            int won = 0;
            if (lane == 0) won = atomicCAS(&T->found, 0, 1) == 0;
            keep = __shfl_sync(FULLMASK, won, 0) != 0;
            stop = 1;
        }
        if (!keep) return;
        const int bit = __ffs(d) - 1;
        const int val = I.lo0 + bit;
        WarpShared &w = ws();
        const int k = w.hcnt;
        if (lane < n) reinterpret_cast<uint8_t *>(&SM[hbuf() + k * HB_STRIDE])[lane] = (uint8_t)bit;
        __syncwarp();
        if (lane == 0) {
            w.sols++;
            w.hcnt = k + 1;
            if (SA.batch) atomicAdd(&SA.results[inst].solutions, 1ull);
        }
        __syncwarp();
        if (k + 1 == HB_SOLS) hash_flush_reg();
        long long slot_off = -1;
        if (SA.mode == 1) {
            slot_off = ws().sol_off;
        } else if (SA.cap > 0) {
            unsigned long long s = 0;
            if (lane == 0 && ld_volatile((const uint32_t *)&SA.g->stored) < (uint32_t)SA.cap)
                s = atomicAdd(&SA.g->stored, 1ull) + 1ull;
            s = __shfl_sync(FULLMASK, s, 0);
            if (s > 0 && (long long)s <= SA.cap) slot_off = (long long)(s - 1) * n;
        }
        if (slot_off >= 0 && SA.sols != nullptr && lane < n) SA.sols[slot_off + lane] = val;
        __syncwarp();
    }

    // unfixed variables of the record at SM offset `Ls` (>= 0) or global `Lg` (every lane)
    __device__ int count_unfixed(int Ls, const uint32_t *Lg) const {
        int c = 0;
        for (int v = lane_id(); v < I.n; v += 32) {
            int p = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) p += __popc(Ls >= 0 ? SM[Ls + v * W + k] : Lg[v * W + k]);
            c += p > 1;
        }
        return __reduce_add_sync(FULLMASK, c);
    }
    __device__ __forceinline__ int ubin(int u) const { return u * UBINS / (I.n + 1); }

    // Donate to waiting workers, shallowest levels (the largest subtrees) first: promise up
    // to `most` records owed to them, at most one per untried value of the level, split the
    // level's values one per record (the last record takes the rest), so that one donation
    // feeds several waiting workers without records hopping from thief to thief.  The level
    // being expanded keeps its lowest value.  A level is not given away when the records
    // with its share of unfixed variables taken so far took little time on average; the
    // levels below it are smaller still, so the donation ends there.
    __device__ __noinline__ void donate(int most) {
        const int lane = lane_id();
        for (int s = 0; s < top; ++s) {
            const bool in_sm = s >= base;
            uint32_t *Lg = in_sm ? nullptr : spill(s);
            const int Ls = in_sm ? slot(s) : -1;
            uint32_t r = 0u;
            if (lane < W) r = in_sm ? SM[Ls + S + lane] : Lg[S + lane];
            int pc = __reduce_add_sync(FULLMASK, __popc(r));
            if (s == top - 1) {                         // keep the lowest value
                const uint32_t nz = __ballot_sync(FULLMASK, r != 0u);
                if (nz && lane == __ffs(nz) - 1) r &= r - 1;
                pc -= nz ? 1 : 0;
            }
            if (pc == 0) continue;
            // the size bin's worth, from the statistics last read (refresh_worth)
            const int u = count_unfixed(Ls, Lg);
            if (!((worth_bins >> ubin(u)) & 1u)) return;
            int budget = 0;
            if (lane == 0) {
                const int k = min(most, pc);
                const uint32_t h = ld_volatile(&T->head);
                const uint32_t p0 = atomicAdd(&T->promised, (uint32_t)k);
                budget = min(max((int)(h - p0), 0), k);
                if (budget < k) atomicSub(&T->promised, (uint32_t)(k - budget));
            }
            budget = __shfl_sync(FULLMASK, budget, 0);
            if (budget == 0) return;                      // nobody is waiting any more
            most -= budget;
            while (budget > 0) {
                // give the highest value alone, or all that is left with the last record
                uint32_t give = r;
                if (budget > 1 && pc > 1) {
                    const uint32_t nz = __ballot_sync(FULLMASK, r != 0u);
                    const int k = 31 - __clz(nz);
                    give = lane == k ? 1u << (31 - __clz(r)) : 0u;
                }
                if (lane == 0) atomicAdd(&T->work, 1);
                if (!q_push(T, qseq(), qrec(), Ls, Lg, R, S, W, true, give)) {
                    if (lane == 0) {                      // queue full: not given
                        atomicSub(&T->work, 1);
                        atomicSub(&T->promised, (uint32_t)budget);
                    }
                    return;
                }
                r &= ~give;
                if (lane < W) {
                    if (in_sm) SM[Ls + S + lane] &= ~give;
                    else Lg[S + lane] &= ~give;
                }
                __syncwarp();
                if (lane == 0) ws().steals++;
                pc -= __reduce_add_sync(FULLMASK, __popc(give));
                --budget;
            }
            if (most == 0) return;
        }
    }

    // ---------------------------------------------------------------- learned brancher

    // number of fixed variables of the node at C (every lane)
    __device__ int count_fixed_lane0(int C) const {
        int c = 0;
        for (int v = lane_id(); v < I.n; v += 32) c += dom_popc<W>(C + v * W) == 1;
        return __reduce_add_sync(FULLMASK, c);
    }

    // mean over the variables of |D| / initial size at the node C (every lane)
    __device__ float mean_rel_size(int C) const {
        const int vfo = (int)I.w(H_OFF_VFEAT);
        float s = 0.f;
        for (int v = lane_id(); v < I.n; v += 32)
            s += (float)dom_popc<W>(C + v * W) / (float)I.w(vfo + VFEAT_WORDS * v + 1);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULLMASK, s, o);
        return s / (float)I.n;
    }

    // The 16 features of variable v at the node C (one lane): domain size, log size, degree,
    // unfixed neighbours, neighbours' relative size, bounds, mean relative domain size of the
    // node, fraction fixed, mix of
    // constraint kinds, mean table tightness, size per unfixed neighbour, bias.
    // Every feature depends only on the node's domains and the model, so the learned choice
    // is the same whichever worker expands the node.
    __device__ void var_features(int C, int v, float mrel, int nfixed, float (&f)[N_FEATURES]) const {
        const int vfo = (int)I.w(H_OFF_VFEAT);
        const int vf = vfo + VFEAT_WORDS * v;
        const int lo_off = (int)I.w(vf), size0 = (int)I.w(vf + 1), deg = (int)I.w(vf + 2);
        const int d = C + v * W;
        const int pc = dom_popc<W>(d), mn = dom_min<W>(d), mx = dom_max<W>(d);
        const int nbs = (int)I.w(H_OFF_NB_START), nbl = (int)I.w(H_OFF_NB);
        const int k0 = (int)I.w(nbs + v), k1 = (int)I.w(nbs + v + 1);
        int unfixed = 0;
        float rel = 0.f;
        for (int k = k0; k < k1; ++k) {
            const int u = (int)I.w(nbl + k);
            const int pu = dom_popc<W>(C + u * W);
            if (pu > 1) {
                unfixed++;
                rel += (float)pu / (float)I.w(vfo + VFEAT_WORDS * u + 1);
            }
        }
        const float s0 = (float)max(size0, 2), span = (float)max(size0 - 1, 1);
        const float dg = (float)max(deg, 1);
        f[0] = (float)pc / s0;
        f[1] = __log2f((float)max(pc, 1)) / __log2f(s0);
        f[2] = (float)deg / (float)I.w(H_MAXDEG);
        f[3] = (float)unfixed / (float)max(k1 - k0, 1);
        f[4] = unfixed ? rel / (float)unfixed : 0.f;
        f[5] = (float)(mn - lo_off) / span;
        f[6] = (float)(mx - lo_off) / span;
        f[7] = mrel;
        f[8] = (float)nfixed / (float)I.n;
        f[9] = (float)I.w(vf + 3) / dg;
        f[10] = (float)I.w(vf + 4) / dg;
        f[11] = (float)I.w(vf + 5) / dg;
        f[12] = (float)I.w(vf + 6) / dg;
        f[13] = __uint_as_float(I.w(vf + 7));
        f[14] = (float)pc / (s0 * (float)(1 + unfixed));
        f[15] = 1.f;
    }

    // The unfixed variable with the smallest predicted log2 subtree size (ties: fewest
    // values, then lowest index).  Falls back to the first-fail choice y_ff when a score is
    // not a number.  Feature rows are staged as bf16 pairs in the warp's tile; the network
    // runs on the tensor cores, 16 variables per mma tile.
    __device__ __noinline__ int select_learned(int C, int y_ff) {
        const int lane = lane_id();
        const int n = I.n;
        const int feat = wso + WS_WORDS;
        const int nfixed = count_fixed_lane0(C);
        const float mrel = mean_rel_size(C);
        const int npad = (n + 15) & ~15;
        for (int v = lane; v < npad; v += 32) {
            float f[N_FEATURES];
            if (v < n) var_features(C, v, mrel, nfixed, f);
#pragma unroll
            for (int j = 0; j < N_FEATURES / 2; ++j)
                SM[feat + v * 8 + j] = v < n ? pack_bf16(f[2 * j], f[2 * j + 1]) : 0u;
        }
        __syncwarp();
        unsigned long long best = ~0ull;
        bool nan = false;
        const int g = lane >> 2;
        for (int r0 = 0; r0 < npad; r0 += 16) {
            auto x = [&](int r, int c) -> uint32_t { return SM[feat + (r0 + r) * 8 + (c >> 1)]; };
            auto pk = [&](int i) -> uint32_t { return SM[SA.mlp_off + i]; };
            float s_lo, s_hi;
            mlp_tile(x, pk, s_lo, s_hi);
            if ((lane & 3) == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int v = r0 + g + 8 * h;
                    const float sc = h ? s_hi : s_lo;
                    if (v < n) {
                        const int pc = dom_popc<W>(C + v * W);
                        if (pc > 1) {
                            if (sc != sc) nan = true;
                            const uint32_t u = __float_as_uint(sc);
                            const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
                            const unsigned long long key =
                                ((unsigned long long)ord << 32) | ((unsigned)pc << 16) | (unsigned)v;
                            best = key < best ? key : best;
                        }
                    }
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(FULLMASK, best, o);
            best = other < best ? other : best;
        }
        if (__any_sync(FULLMASK, nan) || best == ~0ull) return y_ff;
        return (int)(best & 0xffffu);
    }

    // subtree logging: the level at P is complete; its subtree had nodes - start nodes
    __device__ __noinline__ void log_level(int P) {
        if (lane_id() == 0) {
            const uint32_t start = SM[P + S + W + 1];
            const uint32_t size = (uint32_t)ws().nodes - start;
            const uint32_t h = (uint32_t)splitmix64(((unsigned long long)gw << 32) | start);
            if (size > 0 && (SA.log_sample <= 1 || h % SA.log_sample == 0)) {
                const unsigned long long slot = atomicAdd(SA.log_count, 1ull);
                if ((long long)slot < SA.log_cap) {
                    float *e = SA.logbuf + slot * (N_FEATURES + 1);
                    for (int i = 0; i < N_FEATURES; ++i) e[i] = __uint_as_float(SM[P + S + W + 2 + i]);
                    e[N_FEATURES] = __log2f((float)size);
                }
            }
        }
        __syncwarp();
    }

    // propagate the node in the shared slot C of level cl; open a level on success
    __device__ void node(int C, int cl, bool full) {
        const int lane = lane_id();
        tick++;
        // loads whose latency overlaps the fixpoint: stop flags and the donation signal
        const int p_stop = poll();
        uint32_t p_head = 0, p_prom = 0;
        const bool may_donate = donation_due();
        if (may_donate && lane == 0) {
            p_head = ld_volatile(&T->head);
            p_prom = ld_volatile(&T->promised);
        }
        if ((tick & 63) == 0) check_limits();
        unsigned long long ev = 0, rnd = 0;
        const int list = SA.list_words ? wso + WS_WORDS + SA.feat_words : -1;
        const bool failed = fixpoint<W, ST>(I, C, chg(), evs(), full, ev, rnd, list);
        // a root shared by several ranks (its children dealt round-robin) counts on rank 0 only
        const bool split_root = full && !SA.batch && SA.nparts > 1;
        const bool counted = !split_root || SA.part == 0;
        if (lane == 0 && counted) {
            WarpShared &w = ws();
            w.nodes++;
            w.evals += ev;
            w.rounds += rnd;
        }
        stop = __shfl_sync(FULLMASK, p_stop, 0);
        if (failed) {
            if (lane == 0 && counted) ws().fails++;
            refill();
            return;
        }
        int y = select_first_fail<W>(C, I.n);
        if (y < 0) {
            if (counted) record_solution(C);
            refill();
            return;
        }
        if (EXT && SA.mlp_off >= 0) y = select_learned(C, y);
        if (EXT && SA.log_extra) {
            // subtree logging: remember the node count and the chosen variable's features
            float f[N_FEATURES];
            const int nfixed = count_fixed_lane0(C);          // warp-wide reductions
            const float mrel = mean_rel_size(C);
            if (lane == 0) {
                var_features(C, y, mrel, nfixed, f);
                SM[C + S + W + 1] = (uint32_t)ws().nodes;
#pragma unroll
                for (int i = 0; i < N_FEATURES; ++i) SM[C + S + W + 2 + i] = __float_as_uint(f[i]);
            }
            __syncwarp();
        }
        uint32_t rw = lane < W ? SM[C + y * W + lane] : 0u;
        if (split_root) {
            // keep the values whose position in D(y), ascending, is part mod nparts
            uint32_t before = 0;
            for (int k = 0; k < W; ++k) {
                const uint32_t pk = __shfl_sync(FULLMASK, (uint32_t)__popc(rw), k);
                if (k < lane) before += pk;
            }
            uint32_t keep = 0;
            for (uint32_t m = rw; m; m &= m - 1) {
                const uint32_t bit = m & (~m + 1u);
                const uint32_t pos = before + (uint32_t)__popc(rw & (bit - 1u));
                if (pos % (uint32_t)SA.nparts == (uint32_t)SA.part) keep |= bit;
            }
            rw = keep;
        }
        if (lane < W) SM[C + S + lane] = rw;
        if (lane == 0) SM[C + S + W] = (uint32_t)y;
        __syncwarp();
        top = cl + 1;
        if (lane == 0 && top > ws().maxd) ws().maxd = top;
        if (may_donate) {
            // records owed to waiting workers, a bounded number per node
            const int owed = max((int)(p_head - p_prom), 0);
            owed_seen = __shfl_sync(FULLMASK, owed, 0);
            const int want = min(owed_seen, CUBICS_DONATE_MAX);
            hungry = want > 0;
            if (want > 0) donate(want);
        }
    }

    // node() for a node held in registers: d is lane i's D(x_i), `pending` the fixed
    // variables not yet propagated, `done` the ones already propagated (full: the record's
    // root node, whose unary constraints and fixed variables are all still to apply).  On
    // success the node opens level cl in its shared slot.
    __device__ void node_reg(uint32_t d, int cl, uint32_t pending, uint32_t done, bool full,
                             int x = -1, int ax = 0) {
        const int lane = lane_id();
        const int n = I.n;
        tick++;
        const bool polled = full || (tick & (CUBICS_POLL_EVERY - 1u)) == 0u;
        const int p_stop = polled ? poll() : 0;
        uint32_t p_head = 0, p_prom = 0;
        const bool may_donate = donation_due();
        if (may_donate && lane == 0) {
            p_head = ld_volatile(&T->head);
            p_prom = ld_volatile(&T->promised);
        }
        if ((tick & 63) == 0) check_limits();
        unsigned long long ev = 0, rnd = 0;
        bool failed = false;
        if (full) {
            const int nun = (int)I.w(H_N_UN), un = (int)I.w(H_OFF_UN);
            for (int k = 0; k < nun; ++k) {
                const uint32_t u = I.w(un + k);
                if ((int)(u & 0xffffu) == lane) d &= ~(1u << (u >> 16));
            }
            failed = __any_sync(FULLMASK, lane < n && d == 0u);
            pending = __ballot_sync(FULLMASK, lane < n && (d & (d - 1u)) == 0u);
        }
        if (!failed) failed = fixpoint_reg<ST>(I, d, pending, full ? 0u : done, ev, rnd, x, ax);
        const bool split_root = full && !SA.batch && SA.nparts > 1;
        const bool counted = !split_root || SA.part == 0;
        if (counted) {
            cnt_nf += failed ? 0x10001u : 1u;
            cnt_er += (uint32_t)ev | ((uint32_t)rnd << 16);
        }
        if (polled) stop = __shfl_sync(FULLMASK, p_stop, 0);
        if (failed) {
            refill();
            return;
        }
        const int y = select_first_fail_reg(d, n);
        if (y < 0) {
            if (counted) record_solution_reg(d);
            refill();
            return;
        }
        uint32_t rw = __shfl_sync(FULLMASK, d, y);
        if (split_root) {
            // keep the values whose position in D(y), ascending, is part mod nparts
            uint32_t keep = 0;
            for (uint32_t m = rw; m; m &= m - 1) {
                const uint32_t bit = m & (~m + 1u);
                if ((uint32_t)__popc(rw & (bit - 1u)) % (uint32_t)SA.nparts == (uint32_t)SA.part) keep |= bit;
            }
            rw = keep;
        }
        const int C = slot(cl);
        if (lane < n) SM[C + lane] = d;
        if (lane == 0) {
            SM[C + S] = rw;
            SM[C + S + 1] = (uint32_t)y;
        }
        __syncwarp();
        top = cl + 1;
        if (lane == 0 && top > ws().maxd) ws().maxd = top;
        if (may_donate) {
            const int owed = max((int)(p_head - p_prom), 0);
            owed_seen = __shfl_sync(FULLMASK, owed, 0);
            const int want = min(owed_seen, CUBICS_DONATE_MAX);
            hungry = want > 0;
            if (want > 0) donate(want);
        }
    }

    // Solutions of a pair of nodes (expand_pair_reg): bit h of `sol` for node h, whose lanes
    // 16h + i hold the one value of x_i.  The values go to the hash buffer (node 0 first) and,
    // with a cap, to the solution store.
    __device__ __noinline__ void record_solution_pair(uint32_t d, uint32_t sol) {
        const int lane = lane_id();
        const int h = lane >> 4, i = lane & 15;
        const int n = I.n;
        const int ns = __popc(sol);
        WarpShared &w = ws();
        if (w.hcnt + ns > HB_SOLS) hash_flush_reg();
        const int k = w.hcnt;
        const bool mine = (sol >> h) & 1u;
        const int bit = __ffs(d) - 1;
        const int at = k + ((h == 1 && (sol & 1u)) ? 1 : 0);
        if (mine && i < n) reinterpret_cast<uint8_t *>(&SM[hbuf() + at * HB_STRIDE])[i] = (uint8_t)bit;
        __syncwarp();
        if (lane == 0) {
            w.sols += (unsigned long long)ns;
            w.hcnt = k + ns;
            if (SA.batch) atomicAdd(&SA.results[inst].solutions, (unsigned long long)ns);
        }
        __syncwarp();
        if (k + ns == HB_SOLS) hash_flush_reg();
        if (SA.cap > 0 && SA.sols != nullptr) {
            for (int s2 = 0; s2 < 2; ++s2) {
                if (!((sol >> s2) & 1u)) continue;
                unsigned long long t = 0;
                if (lane == 0 && ld_volatile((const uint32_t *)&SA.g->stored) < (uint32_t)SA.cap)
                    t = atomicAdd(&SA.g->stored, 1ull) + 1ull;
                t = __shfl_sync(FULLMASK, t, 0);
                if (t > 0 && (long long)t <= SA.cap && h == s2 && i < n)
                    SA.sols[(long long)(t - 1) * n + i] = I.lo0 + bit;
            }
            __syncwarp();
        }
    }

    // expand_reg for two children at once (all-solution search, n <= 16): the two lowest
    // untried values of the top level, child h in half-warp h (lane 16h + i: D(x_i)).  Each
    // child fails, is a solution or opens a level; child 1's level goes below child 0's, so
    // child 0's subtree is searched first, and every node is still visited once: the counts
    // and hashes are those of the depth-first search.  The stack holds up to two levels per
    // depth (2n - 1 in all; the plan gives it 2n).
    __device__ CUBICS_PAIR_INLINE void expand_pair_reg(int P, int p, uint32_t r) {
        const int lane = lane_id();
        const int h = lane >> 4, i = lane & 15;
        const int n = I.n;
        const int v0 = __ffs(r) - 1;
        const uint32_t r1 = r & (r - 1u);
        const int v1 = __ffs(r1) - 1;
        const uint32_t rest = r1 & (r1 - 1u);
        const int x = (int)SM[P + S + 1];
        const bool act = i < n;
        uint32_t d = act ? SM[P + i] : 0u;
        // the parent is at its fixpoint: its fixed variables' consequences are in d already
        const uint32_t done = __ballot_sync(FULLMASK, act && (d & (d - 1u)) == 0u);
        if (i == x) d = 1u << (h ? v1 : v0);
        int cl;
        if (rest == 0u) {                 // the last two values: the level's slot is reused
            cl = p;
            top = p;
        } else {
            if (lane == 0) SM[P + S] = rest;
            cl = p + 1;
            make_room(cl);
        }
        __syncwarp();
        tick++;
        const bool polled = (tick & (CUBICS_POLL_EVERY - 1u)) == 0u;
        const int p_stop = polled ? poll() : 0;
        uint32_t p_head = 0, p_prom = 0;
        const bool may_donate = donation_due();
        if (may_donate && lane == 0) {
            p_head = ld_volatile(&T->head);
            p_prom = ld_volatile(&T->promised);
        }
        if ((tick & 63) == 0) check_limits();
        uint32_t ev = 0u, rnd = 0u;
        const uint32_t fm = fixpoint_pair_reg<ST>(I, d, x, h ? v1 : v0, done, ev, rnd);
        const uint32_t f = (fm & 1u) | ((fm >> 15) & 2u);          // bit h: node h failed
        cnt_nf += 2u + ((uint32_t)__popc(f) << 16);
        cnt_er += ((ev & 0xffffu) + (ev >> 16)) | (((rnd & 0xffffu) + (rnd >> 16)) << 16);
        if (polled) stop = __shfl_sync(FULLMASK, p_stop, 0);
        uint32_t open = 0u;                                         // bit h: node h branches
        int y = -1;
        if (f != 3u) {                                              // not both failed
            y = select_first_fail_pair(d, n, (f >> h) & 1u);
            const uint32_t yb = __ballot_sync(FULLMASK, i == 0 && y >= 0);
            open = (yb & 1u) | ((yb >> 15) & 2u);
            const uint32_t sol = ~f & ~open & 3u;
            if (sol) record_solution_pair(d, sol);
        }
        if (open) {
            // node 1's level first (at cl, which has room), node 0's above it
            const int l0 = (open & 2u) ? cl + 1 : cl;
            if (open == 3u) make_room(l0);
            const int C = slot(h ? cl : l0);
            const uint32_t rw = __shfl_sync(FULLMASK, d, (lane & 16) + (y < 0 ? 0 : y));
            if ((open >> h) & 1u) {
                if (act) SM[C + i] = d;
                if (i == 0) {
                    SM[C + S] = rw;
                    SM[C + S + 1] = (uint32_t)y;
                }
            }
            __syncwarp();
            top = cl + __popc(open);
            if (lane == 0 && top > ws().maxd) ws().maxd = top;
        } else {
            refill();
        }
        if (may_donate) {
            const int owed = max((int)(p_head - p_prom), 0);
            owed_seen = __shfl_sync(FULLMASK, owed, 0);
            const int want = min(owed_seen, CUBICS_DONATE_MAX);
            hungry = want > 0;
            if (want > 0) donate(want);
        }
    }

    // expand() for register-held nodes: the parent's domains go straight into registers; only
    // a child that opens a level is written back
    __device__ void expand_reg() {
        const int lane = lane_id();
        const int p = top - 1;
        const int P = slot(p);
        const uint32_t r = SM[P + S];
        if (!r) {
            top = p;
            refill();
            return;
        }
        if (SA.pairs && I.n <= 16 && (r & (r - 1u))) {
            expand_pair_reg(P, p, r);
            return;
        }
        const int v = __ffs(r) - 1;
        const uint32_t rest = r & (r - 1u);
        const int x = (int)SM[P + S + 1];
        uint32_t d = lane < I.n ? SM[P + lane] : 0u;
        // the parent is at its fixpoint: its fixed variables' consequences are in d already
        const uint32_t done = __ballot_sync(FULLMASK, lane < I.n && (d & (d - 1u)) == 0u);
        if (lane == x) d = 1u << v;
        __syncwarp();
        int cl;
        if (rest == 0u) {                 // the last value: the level's slot becomes the child's
            cl = p;
            top = p;
        } else {
            if (lane == 0) SM[P + S] = rest;
            cl = p + 1;
            make_room(cl);
        }
        __syncwarp();
        node_reg(d, cl, 1u << x, done, false, x, v);
    }

    // child of the top level: next value of its branching variable (the level is popped
    // when it has none left)
    __device__ void expand() {
        if constexpr (REG) expand_reg();
        else expand_copy();
    }

    __device__ void expand_copy() {
        const int lane = lane_id();
        const int p = top - 1;
        const int P = slot(p);
        const uint32_t r = lane < W ? SM[P + S + lane] : 0u;
        const uint32_t nz = __ballot_sync(FULLMASK, r != 0u);
        if (!nz) {
            if (EXT && SA.log_extra) log_level(P);
            top = p;
            refill();
            return;
        }
        const int k = __ffs(nz) - 1;
        const uint32_t rw = __shfl_sync(FULLMASK, r, k);
        const int v = (k << 5) + __ffs(rw) - 1;
        const uint32_t rest = rw & (rw - 1);
        // the last value reuses the level's slot, unless the level must outlive its last
        // child to measure its subtree
        const bool last = rest == 0u && (nz & ~(1u << k)) == 0u && !(EXT && SA.log_extra);
        const int x = (int)SM[P + S + W];
        int C, cl;
        __syncwarp();
        if (last) {
            cl = p;
            C = P;
            top = p;          // the level is consumed; its slot becomes the child
        } else {
            if (lane == k) SM[P + S + k] = rest;
            cl = p + 1;
            make_room(cl);
            C = slot(cl);
            __syncwarp();
            copy_ss(C, P, R);
        }
        __syncwarp();
        if (lane < W) SM[C + x * W + lane] = (lane == (v >> 5)) ? (1u << (v & 31)) : 0u;
        if (lane < I.NW) SM[chg() + lane] = (lane == (x >> 5)) ? (1u << (x & 31)) : 0u;
        __syncwarp();
        node(C, cl, false);
    }

    // run the record now in slot 0 to exhaustion
    __device__ void explore() {
        base = 0;
        top = 0;
        stop = __shfl_sync(FULLMASK, poll(), 0);
        if (stop) return;
        const int var = (int)SM[slots + S + W];
        if (var < 0) {
            if constexpr (REG) node_reg(lane_id() < I.n ? SM[slots + lane_id()] : 0u, 0, 0u, 0u, true);
            else node(slots, 0, true);
        } else {
            top = 1;
        }
        while (top > 0) {
            if (stop) { top = 0; break; }
            expand();
        }
    }

    // take records until the team has no work left
    __device__ void run() {
        const int lane = lane_id();
        for (;;) {
            uint32_t ticket = 0;
            if (lane == 0) ticket = atomicAdd(&T->head, 1u);
            ticket = __shfl_sync(FULLMASK, ticket, 0);
            const long long t0 = global_ns();
            int got = 0;
            unsigned sleep = 32;
            for (int it = 0;; ++it) {
                if (q_take(qseq(), qrec(), ticket, slots, R)) { got = 1; break; }
                int done = 0;
                if (lane == 0 && (it & 3) == 3) {   // termination and limits, every 4th poll
                    // work == 0: no record is queued or being explored, so none will come;
                    // the ticket is abandoned (the queue is not used again in this launch)
                    if (ld_volatile(&T->work) == 0 || ld_volatile(&SA.g->abort)) done = 1;
                    else if (global_ns() - t0 > SA.wait_limit_ns) {
                        atomicCAS(&SA.g->status, 0, CSP_ETIMEOUT_);
                        atomicExch(&SA.g->abort, 1);
                        done = 1;
                    }
                }
                if (__shfl_sync(FULLMASK, done, 0)) break;
                // jittered so that the waiting workers do not poll in step
                __nanosleep(sleep + ((unsigned)gw * 97u & 511u));
                sleep = sleep < CUBICS_POLL_MAX_NS ? sleep * 2 : CUBICS_POLL_MAX_NS;
            }
            if (lane == 0) ws().wait_ns += global_ns() - t0;
            if (!got) {
                if constexpr (REG) {
                    // before a batch worker moves to another instance (other n and lo0)
                    fold_counts();
                    if (ws().hcnt > 0) hash_flush_reg();
                }
                return;
            }
            taken = tick;
            // the record's size bin (its share of unfixed variables); with running credit,
            // it counts in its bin now and its nodes are credited as they are explored (every
            // 64th node and at the end); otherwise it counts once it has finished
            pbin = ubin(count_unfixed(slots, nullptr));
            credited = tick;
            const long long t_taken = global_ns();
            if (lane == 0 && !CUBICS_FINISHED_STATS) atomicAdd(&T->ucnt[pbin], 1u);
            explore();
            __syncwarp();
            if (lane == 0) {
                if (CUBICS_FINISHED_STATS) atomicAdd(&T->ucnt[pbin], 1u);
                atomicAdd(&T->usum[pbin], (unsigned long long)(tick - credited));
                atomicAdd(&T->xnodes, (unsigned long long)(tick - taken));
                atomicAdd(&T->xns, (unsigned long long)(global_ns() - t_taken));
                __threadfence();
                atomicSub(&T->work, 1);
            }
        }
    }

    __device__ void init_shared() {
        if (lane_id() == 0) {
            WarpShared &w = ws();
            w.nodes = w.fails = w.sols = w.hsum = w.hxor = 0;
            w.evals = w.steals = w.spills = 0;
            w.maxd = 0;
            w.hcnt = 0;
            w.sol_off = 0;
            w.wait_ns = 0;
            w.rounds = 0;
            w.t_start = global_ns();
        }
        __syncwarp();
    }

    __device__ void flush() {
        if constexpr (REG) {
            fold_counts();
            if (ws().hcnt > 0) hash_flush_reg();
        }
        if (lane_id() == 0) {
            GState *g = SA.g;
            WarpShared &w = ws();
            atomicAdd(&g->nodes, w.nodes);
            atomicAdd(&g->fails, w.fails);
            atomicAdd(&g->solutions, w.sols);
            atomicAdd(&g->hsum, w.hsum);
            atomicXor(&g->hxor, w.hxor);
            atomicAdd(&g->evals, w.evals);
            atomicAdd(&g->steals, w.steals);
            atomicAdd(&g->spills, w.spills);
            atomicAdd(&g->wait_ns, (unsigned long long)w.wait_ns);
            atomicAdd(&g->rounds, w.rounds);
            atomicMax(&g->max_depth, w.maxd);
        }
    }
};

// stage an instance's constraint words into SM[0..) (whole block)
__device__ __forceinline__ void stage_instance(const uint32_t *ib) {
    const int words = ((int)ib[H_CONS_WORDS] + 3) & ~3;
    const uint4 *s = reinterpret_cast<const uint4 *>(ib);
    uint4 *d = reinterpret_cast<uint4 *>(SM);
    for (int i = threadIdx.x; i < words / 4; i += blockDim.x) d[i] = s[i];
}

template <int W, bool ST, bool EXT, bool REG = false>
__device__ __forceinline__ void search_body(const SearchArgs &Ap) {
    const int warp = threadIdx.x >> 5, lane = lane_id();
    __shared__ int s_inst, s_team;
    if (threadIdx.x == 0) SA = Ap;
    __syncthreads();
    if (REG && SA.hash_words < HB_WORDS) {      // no room for the deferred solution hashes
        if (threadIdx.x == 0) atomicCAS(&SA.g->status, 0, CSP_EINVAL_);
        return;
    }
    const int per_warp = SA.lsm * SA.rmax + WS_WORDS + SA.feat_words + SA.list_words + SA.hash_words;
    if (EXT && SA.mlp_off >= 0) {    // the brancher's weights, staged once per block
        for (int i = threadIdx.x; i < PK_WORDS; i += blockDim.x) SM[SA.mlp_off + i] = __ldg(SA.mlp + i);
        __syncthreads();
    }

    Worker<W, ST, EXT, REG> wk;
    wk.lsm = SA.lsm;
    wk.slots = SA.warp_base + warp * per_warp;
    wk.wso = wk.slots + SA.lsm * SA.rmax;
    wk.gw = blockIdx.x * SA.warps + warp;
    wk.tick = 0;
    wk.hungry = 1;                   // the first nodes feed the idle workers at once
    wk.worth_bins = 0xffffffffu;     // nothing observed yet: every size is worth passing on
    wk.owed_seen = 0;
    wk.taken = 0;
    wk.pbin = 0;
    wk.credited = 0;
    wk.stop = 0;
    wk.cnt_nf = wk.cnt_er = 0u;
    wk.team = 0;
    wk.inst = 0;
    wk.init_shared();

    if (!SA.batch) {
        const uint32_t *ib = SA.arena + SA.inst_off[0];
        if (ST) stage_instance(ib);
        __syncthreads();
        wk.I.load(ib);
        wk.S = wk.I.S;
        wk.R = record_words(wk.S, W, SA.log_extra);
        wk.T = SA.teams;
        wk.run();
        wk.flush();
        return;
    }

    // Batch mode.  A block takes instance tickets and is the team of each instance it owns;
    // once the tickets are gone it joins teams whose instance is still being searched
    // (stages that instance and takes records from the team's queue), so the last, hardest
    // instances are shared by every block.
    for (;;) {
        if (threadIdx.x == 0) {
            const bool aborted = ld_volatile(&SA.g->abort) != 0;
            int t = aborted ? SA.n_inst : atomicAdd(&SA.g->ticket, 1);
            int team = blockIdx.x;
            if (t >= SA.n_inst) {
                t = -1;
                team = -1;
                // helpers can only take donated work: no joining when donation is off
                const bool join = !aborted && !(SA.flags & F_NO_DONATE);
                for (int k = 1; join && k <= (int)gridDim.x; ++k) {
                    const int c = (blockIdx.x + k) % gridDim.x;
                    Team *Tc = SA.teams + c;
                    if (ld_volatile(&Tc->work) > 0) {
                        // counted among the team's helpers before the instance is read: the
                        // owner does not reuse the queue for its next instance while helpers
                        // may hold tickets of this one
                        atomicAdd(&Tc->helpers, 1);
                        __threadfence();
                        if (ld_volatile(&Tc->work) > 0) {
                            __threadfence();
                            t = ld_volatile(&Tc->inst);
                            team = c;
                            break;
                        }
                        atomicSub(&Tc->helpers, 1);
                    }
                }
            }
            s_inst = t;
            s_team = team;
        }
        __syncthreads();
        const int i = s_inst, team = s_team;
        if (i < 0 || i >= SA.n_inst) break;
        const bool own = team == (int)blockIdx.x;
        Team *T = SA.teams + team;
        const uint32_t *ib = SA.arena + SA.inst_off[i];
        if (ST) stage_instance(ib);
        __syncthreads();
        wk.I.load(ib);
        wk.S = wk.I.S;
        wk.R = record_words(wk.S, W, SA.log_extra);
        wk.T = T;
        wk.worth_bins = 0xffffffffu;     // another team: its statistics are read at the next check
        wk.team = team;
        wk.inst = i;
        const unsigned long long n0 = wk.ws().nodes, f0 = wk.ws().fails;
        if (lane == 0) wk.ws().sol_off = SA.sol_off ? SA.sol_off[i] : 0;
        __syncwarp();
        if (own && warp == 0) {
            // root record: the instance's root domains, nothing to try yet, var = -1
            const uint32_t *root = SA.roots ? SA.roots + (size_t)i * wk.S : ib + ib[H_OFF_ROOT];
            for (int k = lane; k < wk.R; k += 32)
                SM[wk.slots + k] = k < wk.S ? root[k] : (k == wk.S + W ? 0xffffffffu : 0u);
            if (lane == 0) {
                // The block's workers abandoned their tickets when the previous instance
                // ended, and so do the helpers of other blocks, which leave once they see
                // work == 0.  Ticket numbers restart at the tail: the queue is reused only
                // when no helper is left (a stale ticket equal to a new one would take the
                // new root too).  Bounded wait: past the wait limit the launch stops with
                // CSP_ETIMEOUT.
                const long long w0 = global_ns();
                for (int it = 0; ld_volatile(&T->helpers) > 0; ++it) {
                    if (it >= (1 << 24) || global_ns() - w0 > SA.wait_limit_ns) {
                        atomicCAS(&SA.g->status, 0, CSP_ETIMEOUT_);
                        atomicExch(&SA.g->abort, 1);
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
                const uint32_t t = ld_volatile(&T->tail);
                T->head = t;
                T->promised = t + 1u;                       // the root record, pushed below
                for (int b = 0; b < UBINS; ++b) {
                    T->ucnt[b] = 0u;
                    T->usum[b] = 0ull;
                }
                T->xns = T->xnodes = 0ull;
                T->inst = i;
                T->found = 0;
                T->progress = 0;
                SA.results[i].t_start = global_ns();
                __threadfence();
                atomicExch(&T->work, 1);
            }
            __syncwarp();
            __threadfence();
            q_push(T, wk.qseq(), wk.qrec(), wk.slots, nullptr, wk.R, wk.S, W, false, 0u);
        }
        __syncthreads();
        wk.run();
        if (lane == 0) {
            atomicAdd(&SA.results[i].nodes, wk.ws().nodes - n0);
            atomicAdd(&SA.results[i].fails, wk.ws().fails - f0);
        }
        __syncthreads();
        if (!own && threadIdx.x == 0) {          // every warp of this helper block has left
            __threadfence();
            atomicSub(&T->helpers, 1);
        }
        if (own && threadIdx.x == 0) {
            // every record of the instance is finished (work == 0): its verdict is final
            InstResult &r = SA.results[i];
            const int st = ld_volatile(&SA.g->status);
            __threadfence();
            const unsigned long long sols = *(volatile unsigned long long *)&r.solutions;
            const int fnd = ld_volatile(&T->found);
            // FIRST: a solution settles the verdict.  ALL: an instance stopped at its node limit
            // has an incomplete count, so it is undecided even if it found solutions.
            r.status = fnd == 1 ? 1 : fnd == 2 ? CSP_ELIMIT_ : sols > 0 ? 1 : (st != 0 ? st : 0);
            r.n = (int)ib[H_N];
            r.sol_offset = SA.sol_off ? SA.sol_off[i] : 0;
            r.t_end = global_ns();
        }
        __syncthreads();
    }
    wk.flush();
}

// Register caps of the plain search kernel (first-fail, no logging), the lowest at which it
// compiles without spills for its staged form: 80 registers for one-word domains (24
// resident warps per SM), 96 for wider ones (20).
#ifndef CUBICS_REGS_W1
#define CUBICS_REGS_W1 80
#endif
#ifndef CUBICS_REGS_WN
#define CUBICS_REGS_WN 96
#endif

template <int W, bool ST>
__global__ void __maxnreg__(W == 1 ? CUBICS_REGS_W1 : CUBICS_REGS_WN)
    search_kernel(const SearchArgs Ap) {
    search_body<W, ST, false>(Ap);
}

// learned brancher and/or subtree logging
template <int W, bool ST>
__global__ void __launch_bounds__(512, 1) search_kernel_ext(const SearchArgs Ap) {
    search_body<W, ST, true>(Ap);
}

// one-word int_ne problems of at most 32 variables, domains in registers (FLAG_NE_REG)
#ifndef CUBICS_REGS_REG
#define CUBICS_REGS_REG 64
#endif
template <bool ST>
__global__ void __maxnreg__(CUBICS_REGS_REG) search_kernel_reg(const SearchArgs Ap) {
    search_body<1, ST, false, true>(Ap);
}

// ------------------------------------------------------------------ propagate kernel

template <int W, bool ST>
__global__ void __launch_bounds__(256) propagate_kernel(PropArgs P) {
    if (ST) stage_instance(P.inst);
    __syncthreads();
    IV<ST> I;
    I.load(P.inst);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int warps = blockDim.x >> 5;
    const int S4 = (I.S + 3) & ~3;
    const int dom = P.stage_words + warp * (S4 + 64);
    const int chg = dom + S4, evs = chg + 32;
    unsigned long long evals = 0;
    for (int s = blockIdx.x * warps + warp; s < P.count; s += gridDim.x * warps) {
        const uint32_t *src = P.din + (size_t)s * I.S;
        for (int k = lane; k < I.S; k += 32) SM[dom + k] = src[k];
        __syncwarp();
        unsigned long long rounds = 0;
        const bool failed = fixpoint<W, ST>(I, dom, chg, evs, true, evals, rounds);
        __syncwarp();
        uint32_t *dst = P.dout + (size_t)s * I.S;
        for (int k = lane; k < I.S; k += 32) dst[k] = SM[dom + k];
        if (lane == 0) P.failed[s] = failed ? 1 : 0;
        __syncwarp();
    }
}

// One fixpoint per state, a whole block per state (constraint-parallel propagation of one
// node by all the block's warps).  Shared memory: the staged instance, then the state
// (S words, rounded to 4), its changed set and event set (32 words each).
template <int W, bool ST>
__global__ void __launch_bounds__(1024) propagate_block_kernel(PropArgs P) {
    if (ST) stage_instance(P.inst);
    __syncthreads();
    IV<ST> I;
    I.load(P.inst);
    const int S4 = (I.S + 3) & ~3;
    const int dom = P.stage_words, chg = dom + S4, evs = chg + 32;
    unsigned long long evals = 0, rounds = 0;
    for (int s = blockIdx.x; s < P.count; s += gridDim.x) {
        const uint32_t *src = P.din + (size_t)s * I.S;
        for (int k = threadIdx.x; k < I.S; k += blockDim.x) SM[dom + k] = src[k];
        __syncthreads();
        const bool failed = fixpoint_block<W, ST>(I, dom, chg, evs, true, evals, rounds);
        __syncthreads();
        uint32_t *dst = P.dout + (size_t)s * I.S;
        for (int k = threadIdx.x; k < I.S; k += blockDim.x) dst[k] = SM[dom + k];
        if (threadIdx.x == 0) P.failed[s] = failed ? 1 : 0;
        __syncthreads();
    }
}

// One level of the depth-k split of a single problem, in three passes over the propagated
// states (a warp per state in the first and last).  A failed state is a node and a fail; a
// state with every variable fixed is a unit as it stands (its node is counted when the unit
// is searched); any other state is a node whose first-fail variable (fewest values, lowest
// index) gives one child per value, ascending.  Children and units keep the order of their
// parents (an exclusive scan of the per-state counts places them), so the units of a split
// come out in the same order at every run: the order of a depth-first search.

// first-fail branching variable of a state and its number of values; y = -1 when every
// variable is fixed
template <int W>
__device__ __forceinline__ void branch_of(const uint32_t *st, int n, int &y, int &c) {
    unsigned best = 0xffffffffu;
    for (int v = lane_id(); v < n; v += 32) {
        int pc = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) pc += __popc(st[v * W + k]);
        if (pc > 1) best = min(best, ((unsigned)pc << 16) | (unsigned)v);
    }
    best = __reduce_min_sync(FULLMASK, best);
    y = best == 0xffffffffu ? -1 : (int)(best & 0xffffu);
    c = best == 0xffffffffu ? 0 : (int)(best >> 16);
}

// pass 1: off[s] = children of state s (low 32 bits) | 1 << 32 if it is a unit; nodes and
// fails counted
template <int W>
__global__ void __launch_bounds__(256) expand_count_kernel(ExpandArgs E) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = (int)E.inst[H_N], S = (int)E.inst[H_S];
    for (int s = warp; s < E.count; s += nwarps) {
        if (E.failed[s]) {
            if (lane == 0) {
                atomicAdd(&E.ctr[2], 1ull);
                atomicAdd(&E.ctr[3], 1ull);
                E.off[s] = 0ull;
            }
            continue;
        }
        int y, c;
        branch_of<W>(E.states + (size_t)s * S, n, y, c);
        if (lane == 0) {
            if (y >= 0) atomicAdd(&E.ctr[2], 1ull);
            E.off[s] = y < 0 ? (1ull << 32) : (unsigned long long)c;
        }
    }
}

// pass 2 (one block of 1024 threads): exclusive scan of off[0 .. count); then the level's
// children (ctr[0]) and the units so far (ctr[1], the level's first unit slot in ctr[5]), or
// the overflow flag (ctr[4]) when the children or the units would not fit.  A state has at
// most 256 children and a level at most 2^31 / 256 states, so the packed halves never carry.
template <int W>
__global__ void __launch_bounds__(1024) expand_scan_kernel(ExpandArgs E) {
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int per = (E.count + 1023) / 1024;
    const int b = min(E.count, t * per), e = min(E.count, b + per);
    unsigned long long sum = 0ull;
    for (int i = b; i < e; ++i) sum += E.off[i];
    unsigned long long x = sum;                      // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {                                  // inclusive scan of the warp totals
        unsigned long long w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULLMASK, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    unsigned long long run = x - sum + (wid > 0 ? wsum[wid - 1] : 0ull);
    for (int i = b; i < e; ++i) {
        const unsigned long long v = E.off[i];
        E.off[i] = run;
        run += v;
    }
    if (t == 1023) {
        const unsigned long long children = wsum[31] & 0xffffffffull, units = wsum[31] >> 32;
        const unsigned long long u0 = E.ctr[1];
        if ((long long)children > E.next_cap || (long long)(u0 + units) > E.units_cap) {
            E.ctr[4] = 1ull;
        } else {
            E.ctr[0] = children;
            E.ctr[1] = u0 + units;
            E.ctr[5] = u0;
        }
    }
}

// pass 3: every child and unit written at its place (nothing when the level overflowed)
template <int W>
__global__ void __launch_bounds__(256) expand_write_kernel(ExpandArgs E) {
    if (*(volatile unsigned long long *)&E.ctr[4]) return;
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = (int)E.inst[H_N], S = (int)E.inst[H_S];
    const unsigned long long u0 = E.ctr[5];
    for (int s = warp; s < E.count; s += nwarps) {
        if (E.failed[s]) continue;
        const uint32_t *st = E.states + (size_t)s * S;
        int y, c;
        branch_of<W>(st, n, y, c);
        const unsigned long long o = E.off[s];
        if (y < 0) {
            uint32_t *u = E.units + (size_t)(u0 + (o >> 32)) * S;
            for (int k = lane; k < S; k += 32) u[k] = st[k];
            continue;
        }
        const unsigned long long base = o & 0xffffffffull;
        long long j = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint32_t m = st[y * W + w];
            while (m) {
                const uint32_t bit = m & (~m + 1u);
                m ^= bit;
                uint32_t *ch = E.next + (size_t)(base + j) * S;
                for (int k = lane; k < S; k += 32) {
                    uint32_t val = st[k];
                    if (k >= y * W && k < (y + 1) * W) val = k == y * W + w ? bit : 0u;
                    ch[k] = val;
                }
                ++j;
            }
        }
    }
}

// ------------------------------------------------------------------ host launchers

template <typename K>
cudaError_t launch_k(K kern, const SearchArgs &A, int blocks, int threads, size_t smem,
                     cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, st>>>(A);
    return cudaGetLastError();
}

template <typename K>
cudaError_t occupancy_k(K kern, int threads, size_t smem, int *bps) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (threads > fa.maxThreadsPerBlock) {   // the register cap admits no block this large
        *bps = 0;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, kern, threads, smem);
}

#define CUBICS_DEFINE_REG                                                                    \
    cudaError_t launch_search_reg(bool st_, const SearchArgs &A, int b, int t, size_t sm,     \
                                  cudaStream_t s) {                                         \
        return st_ ? launch_k(search_kernel_reg<true>, A, b, t, sm, s)                      \
                   : launch_k(search_kernel_reg<false>, A, b, t, sm, s);                    \
    }                                                                                       \
    cudaError_t occupancy_reg(bool st_, int t, size_t sm, int *bps) {                       \
        return st_ ? occupancy_k(search_kernel_reg<true>, t, sm, bps)                       \
                   : occupancy_k(search_kernel_reg<false>, t, sm, bps);                     \
    }

template <int W, bool ST, bool EXT>
cudaError_t launch_search_t(const SearchArgs &A, int blocks, int threads, size_t smem,
                            cudaStream_t st) {
    if constexpr (EXT) return launch_k(search_kernel_ext<W, ST>, A, blocks, threads, smem, st);
    else return launch_k(search_kernel<W, ST>, A, blocks, threads, smem, st);
}

template <int W, bool ST, bool EXT>
cudaError_t occupancy_t(int threads, size_t smem, int *bps) {
    if constexpr (EXT) return occupancy_k(search_kernel_ext<W, ST>, threads, smem, bps);
    else return occupancy_k(search_kernel<W, ST>, threads, smem, bps);
}

template <int W, bool ST>
cudaError_t launch_prop_t(const PropArgs &P, int blocks, int threads, size_t smem, cudaStream_t st,
                          bool block_per_node) {
    if (block_per_node) {
        cudaError_t e = cudaFuncSetAttribute(propagate_block_kernel<W, ST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        propagate_block_kernel<W, ST><<<blocks, threads, smem, st>>>(P);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(propagate_kernel<W, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    propagate_kernel<W, ST><<<blocks, threads, smem, st>>>(P);
    return cudaGetLastError();
}

// Two translation units per W (so that they compile in parallel): one defines the plain
// search kernels and the propagate kernels, the other the search kernels with the learned
// brancher and logging; each for both staging modes.
#define CUBICS_DEFINE_SEARCH(WW, EXT, SFX)                                                   \
    cudaError_t launch_search##SFX##_w##WW(bool st_, const SearchArgs &A, int b, int t,     \
                                           size_t sm, cudaStream_t s) {                     \
        return st_ ? launch_search_t<WW, true, EXT>(A, b, t, sm, s)                         \
                   : launch_search_t<WW, false, EXT>(A, b, t, sm, s);                       \
    }                                                                                       \
    cudaError_t occupancy##SFX##_w##WW(bool st_, int t, size_t sm, int *bps) {              \
        return st_ ? occupancy_t<WW, true, EXT>(t, sm, bps)                                 \
                   : occupancy_t<WW, false, EXT>(t, sm, bps);                               \
    }

#define CUBICS_DEFINE_WIDTH(WW)                                                              \
    CUBICS_DEFINE_SEARCH(WW, false, )                                                        \
    cudaError_t launch_expand_w##WW(const ExpandArgs &E, int blocks, cudaStream_t s) {       \
        expand_count_kernel<WW><<<blocks, 256, 0, s>>>(E);                                  \
        expand_scan_kernel<WW><<<1, 1024, 0, s>>>(E);                                       \
        expand_write_kernel<WW><<<blocks, 256, 0, s>>>(E);                                  \
        return cudaGetLastError();                                                          \
    }                                                                                       \
    cudaError_t launch_prop_w##WW(bool st_, const PropArgs &P, int b, int t, size_t sm,     \
                                  cudaStream_t s, bool bpn) {                               \
        return st_ ? launch_prop_t<WW, true>(P, b, t, sm, s, bpn)                           \
                   : launch_prop_t<WW, false>(P, b, t, sm, s, bpn);                         \
    }

#define CUBICS_DEFINE_WIDTH_EXT(WW) CUBICS_DEFINE_SEARCH(WW, true, _ext)

}  // namespace cubics
