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
#include <cuda_runtime.h>
#include "device.cuh"

namespace cubics {

constexpr int CSP_ELIMIT_ = -5;
constexpr int CSP_ETIMEOUT_ = -6;
constexpr int F_NO_DONATE = 1;

// per-warp bookkeeping kept in shared memory (lane 0 writes the counters)
struct WarpShared {
    uint32_t chg[32], evs[32];
    unsigned long long nodes, fails, sols, hsum, hxor, evals, steals, spills;
    long long t_start;
    int64_t sol_off;
    int32_t maxd, pad[3];
};
static_assert(sizeof(WarpShared) == 4 * WS_WORDS, "WarpShared size must match WS_WORDS");

// ------------------------------------------------------------------ work queue
// Bounded multi-producer multi-consumer ring (per-slot sequence numbers).  Lane 0 claims a
// position; the warp copies the record; a release store of the sequence publishes it.

__device__ bool q_push(const SearchArgs &A, Team *T, uint32_t *seq, uint32_t *rec,
                       const uint32_t *src, int R, int S, int W, bool override_rem,
                       uint32_t my_rem) {
    const int lane = lane_id();
    uint32_t pos = 0;
    int ok = 0;
    if (lane == 0) {
        pos = ld_volatile(&T->tail);
        for (int it = 0; it < 256; ++it) {
            const uint32_t s = ld_acquire(&seq[pos & A.qmask]);
            const int dif = (int)(s - pos);
            if (dif == 0) {
                const uint32_t prev = atomicCAS(&T->tail, pos, pos + 1);
                if (prev == pos) { ok = 1; break; }
                pos = prev;
            } else if (dif < 0) {
                break;                               // full
            } else {
                pos = ld_volatile(&T->tail);
            }
        }
    }
    ok = __shfl_sync(FULLMASK, ok, 0);
    if (!ok) return false;
    pos = __shfl_sync(FULLMASK, pos, 0);
    uint32_t *dst = rec + (size_t)(pos & A.qmask) * A.rmax;
    warp_copy4(dst, src, R);
    __syncwarp();
    if (override_rem && lane < W) dst[S + lane] = my_rem;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(&seq[pos & A.qmask], pos + 1);
    return true;
}

__device__ bool q_pop(const SearchArgs &A, Team *T, uint32_t *seq, uint32_t *rec, uint32_t *dst,
                      int R) {
    const int lane = lane_id();
    uint32_t pos = 0;
    int ok = 0;
    if (lane == 0) {
        pos = ld_volatile(&T->head);
        for (int it = 0; it < 256; ++it) {
            const uint32_t s = ld_acquire(&seq[pos & A.qmask]);
            const int dif = (int)(s - (pos + 1));
            if (dif == 0) {
                const uint32_t prev = atomicCAS(&T->head, pos, pos + 1);
                if (prev == pos) { ok = 1; break; }
                pos = prev;
            } else if (dif < 0) {
                break;                               // empty
            } else {
                pos = ld_volatile(&T->head);
            }
        }
    }
    ok = __shfl_sync(FULLMASK, ok, 0);
    if (!ok) return false;
    pos = __shfl_sync(FULLMASK, pos, 0);
    __threadfence();
    warp_copy4_cg(dst, rec + (size_t)(pos & A.qmask) * A.rmax, R);
    __syncwarp();
    __threadfence();
    if (lane == 0) st_release(&seq[pos & A.qmask], pos + A.qmask + 1);
    return true;
}

// ------------------------------------------------------------------ worker

template <int W>
struct Worker {
    const SearchArgs *A;  // shared-memory copy of the launch arguments
    IV I;
    Team *T;
    uint32_t *slots;      // lsm records in shared memory
    WarpShared *ws;
    int lsm, R, S;
    int top, base;        // open levels [0, top); levels >= base are in shared memory
    uint32_t tick;        // nodes of this worker (low bits pace the periodic checks)
    int gw;               // global worker index

    __device__ uint32_t *qseq() const {
        return A->qseq + (A->batch ? (size_t)blockIdx.x * (A->qmask + 1) : 0);
    }
    __device__ uint32_t *qrec() const {
        return A->qrec + (A->batch ? (size_t)blockIdx.x * (A->qmask + 1) * A->rmax : 0);
    }
    __device__ uint32_t *spill() const { return A->spill + (size_t)gw * A->depth * A->rmax; }
    __device__ uint32_t *level(int k) const {
        return k >= base ? slots + (k % lsm) * R : spill() + (size_t)k * R;
    }
    // make the shared slot of level k (== top) free
    __device__ void make_room(int k) {
        const int old = k - lsm;
        if (old >= base) {
            warp_copy4(spill() + (size_t)old * R, slots + (old % lsm) * R, R);
            __syncwarp();
            base = old + 1;
            if (lane_id() == 0) ws->spills++;
        }
    }
    // after a pop: the new top level must be in shared memory
    __device__ void refill() {
        if (top > 0 && top - 1 < base) {
            const int k = top - 1;
            warp_copy4(slots + (k % lsm) * R, spill() + (size_t)k * R, R);
            __syncwarp();
            base = k;
        }
    }

    __device__ bool stopped() const {
        if (A->mode == 1 && ld_volatile(&T->found)) return true;
        return ld_volatile(&A->g->abort) != 0;
    }

    __device__ void check_limits() {
        if (threadIdx.x % 32 == 0) {
            if (A->node_limit > 0) {
                const unsigned long long tot =
                    atomicAdd(&A->g->node_progress, 64ull) + 64ull;
                if ((long long)tot >= A->node_limit) {
                    atomicCAS(&A->g->status, 0, CSP_ELIMIT_);
                    atomicExch(&A->g->abort, 1);
                }
            }
            if (A->deadline_ns > 0 && global_ns() - ws->t_start > A->deadline_ns) {
                atomicCAS(&A->g->status, 0, CSP_ELIMIT_);
                atomicExch(&A->g->abort, 1);
            }
        }
    }

    __device__ void record_solution(const uint32_t *st) {
        const int lane = lane_id();
        const int n = I.n;
        bool keep = true;
        if (A->mode == 1) {
            int won = 0;
            if (lane == 0) won = atomicCAS(&T->found, 0, 1) == 0;
            keep = __shfl_sync(FULLMASK, won, 0) != 0;
        }
        if (!keep) return;
        if (lane == 0) {
            unsigned long long h = 0x9E3779B97F4A7C15ull;
            for (int i = 0; i < n; ++i) {
                const unsigned val = (unsigned)(I.lo0 + dom_min<W>(st + i * W));
                h = splitmix64(h ^ (((unsigned long long)(unsigned)i << 32) | val));
            }
            ws->sols++;
            ws->hsum += h;
            ws->hxor ^= h;
        }
        int64_t slot = -1;
        if (A->mode == 1) {
            slot = ws->sol_off;
        } else if (A->cap > 0) {
            unsigned long long s = 0;
            if (lane == 0 && ld_volatile((const uint32_t *)&A->g->stored) < (uint32_t)A->cap)
                s = atomicAdd(&A->g->stored, 1ull) + 1ull;
            s = __shfl_sync(FULLMASK, s, 0);
            if (s > 0 && (long long)s <= A->cap) slot = (int64_t)(s - 1) * n;
        }
        if (slot >= 0 && A->sols != nullptr)
            for (int i = lane; i < n; i += 32) A->sols[slot + i] = I.lo0 + dom_min<W>(st + i * W);
        __syncwarp();
    }

    // donate the shallowest untried values when another worker is idle
    __device__ void maybe_donate() {
        const int lane = lane_id();
        int want = 0;
        if (lane == 0) {
            const int idle = ld_volatile(&T->idle);
            if (idle > 0) {
                const uint32_t qn = ld_volatile(&T->tail) - ld_volatile(&T->head);
                want = (int)qn < idle;
            }
        }
        if (!__shfl_sync(FULLMASK, want, 0)) return;
        for (int s = 0; s < top; ++s) {
            uint32_t *L = level(s);
            const uint32_t r = lane < W ? L[S + lane] : 0u;
            const int pc = __reduce_add_sync(FULLMASK, __popc(r));
            if (pc == 0) continue;
            if (s == top - 1 && pc < 2) return;
            // the top level keeps its lowest value; a deeper level gives all of them away
            uint32_t give = r;
            if (s == top - 1) {
                const uint32_t nz = __ballot_sync(FULLMASK, r != 0u);
                const int k0 = __ffs(nz) - 1;
                if (lane == k0) give = r & (r - 1);
            }
            if (lane == 0) atomicAdd(&T->work, 1);
            if (q_push(*A, T, qseq(), qrec(), L, R, S, W, true, give)) {
                if (lane < W) L[S + lane] = r & ~give;
                __syncwarp();
                if (lane == 0) ws->steals++;
            } else if (lane == 0) {
                atomicSub(&T->work, 1);
            }
            return;
        }
    }

    // child of the top level: next value of its branching variable; returns false when
    // the level is exhausted (it is popped)
    __device__ bool expand() {
        const int lane = lane_id();
        const int p = top - 1;
        uint32_t *P = level(p);
        const uint32_t r = lane < W ? P[S + lane] : 0u;
        const uint32_t nz = __ballot_sync(FULLMASK, r != 0u);
        if (!nz) {
            top = p;
            refill();
            return false;
        }
        const int k = __ffs(nz) - 1;
        const uint32_t rw = __shfl_sync(FULLMASK, r, k);
        const int v = (k << 5) + __ffs(rw) - 1;
        const uint32_t rest = rw & (rw - 1);
        const bool last = rest == 0u && (nz & ~(1u << k)) == 0u;
        const int x = (int)P[S + W];
        uint32_t *C;
        int cl;
        __syncwarp();
        if (last) {
            cl = p;
            C = P;
            top = p;          // the level is consumed; its slot becomes the child
        } else {
            if (lane == k) P[S + k] = rest;
            cl = p + 1;
            make_room(cl);
            C = slots + (cl % lsm) * R;
            __syncwarp();
            warp_copy4(C, P, R);
        }
        __syncwarp();
        if (lane < W) C[x * W + lane] = (lane == (v >> 5)) ? (1u << (v & 31)) : 0u;
        if (lane < I.NW) ws->chg[lane] = (lane == (x >> 5)) ? (1u << (x & 31)) : 0u;
        __syncwarp();
        node(C, cl, false);
        return true;
    }

    // propagate the node held in the shared slot of level cl; open a level on success
    __device__ void node(uint32_t *C, int cl, bool full) {
        const int lane = lane_id();
        tick++;
        if ((tick & 63) == 0) check_limits();
        unsigned long long ev = 0;
        const bool failed = fixpoint<W>(I, C, ws->chg, ws->evs, full, ev);
        if (lane == 0) { ws->nodes++; ws->evals += ev; }
        if (failed) {
            if (lane == 0) ws->fails++;
            refill();
            return;
        }
        const int y = select_first_fail<W>(C, I.n);
        if (y < 0) {
            record_solution(C);
            refill();
            return;
        }
        if (lane < W) C[S + lane] = C[y * W + lane];
        if (lane == 0) C[S + W] = (uint32_t)y;
        __syncwarp();
        top = cl + 1;
        if (lane == 0 && top > ws->maxd) ws->maxd = top;
        if (!(A->flags & F_NO_DONATE) && (tick & 3) == 0) maybe_donate();
    }

    // run the record now in slot 0 to exhaustion
    __device__ void explore() {
        base = 0;
        uint32_t *L0 = slots;
        const int var = (int)L0[S + W];
        top = 0;
        if (stopped()) return;
        if (var < 0) {
            node(L0, 0, true);
        } else {
            top = 1;
        }
        while (top > 0) {
            if (stopped()) { top = 0; break; }
            expand();
        }
    }

    // take records until the team has no work left
    __device__ void run() {
        const int lane = lane_id();
        for (;;) {
            if (lane == 0) atomicAdd(&T->idle, 1);
            const long long t0 = global_ns();
            int got = 0;
            unsigned sleep = 32;
            for (;;) {
                if (q_pop(*A, T, qseq(), qrec(), slots, R)) { got = 1; break; }
                int done = 0;
                if (lane == 0) {
                    if (ld_volatile(&T->work) == 0 || ld_volatile(&A->g->abort)) done = 1;
                    else if (global_ns() - t0 > A->wait_limit_ns) {
                        atomicCAS(&A->g->status, 0, CSP_ETIMEOUT_);
                        atomicExch(&A->g->abort, 1);
                        done = 1;
                    }
                }
                if (__shfl_sync(FULLMASK, done, 0)) break;
                __nanosleep(sleep);
                sleep = sleep < 4096 ? sleep * 2 : 4096;
            }
            if (lane == 0) atomicSub(&T->idle, 1);
            if (!got) return;
            explore();
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicSub(&T->work, 1);
            }
        }
    }

    __device__ void init_shared() {
        if (lane_id() == 0) {
            ws->nodes = ws->fails = ws->sols = ws->hsum = ws->hxor = 0;
            ws->evals = ws->steals = ws->spills = 0;
            ws->maxd = 0;
            ws->sol_off = 0;
            ws->t_start = global_ns();
        }
        __syncwarp();
    }

    __device__ void flush() {
        if (lane_id() == 0) {
            GState *g = A->g;
            atomicAdd(&g->nodes, ws->nodes);
            atomicAdd(&g->fails, ws->fails);
            atomicAdd(&g->solutions, ws->sols);
            atomicAdd(&g->hsum, ws->hsum);
            atomicXor(&g->hxor, ws->hxor);
            atomicAdd(&g->evals, ws->evals);
            atomicAdd(&g->steals, ws->steals);
            atomicAdd(&g->spills, ws->spills);
            atomicMax(&g->max_depth, ws->maxd);
        }
    }
};

// stage an instance's constraint words into shared memory (whole block)
__device__ const uint32_t *stage_instance(const uint32_t *ib, uint32_t *stage, int stage_words) {
    const int words = ((int)ib[H_CONS_WORDS] + 3) & ~3;
    if (words > stage_words) return ib;
    const uint4 *s = (const uint4 *)ib;
    uint4 *d = (uint4 *)stage;
    for (int i = threadIdx.x; i < words / 4; i += blockDim.x) d[i] = s[i];
    return stage;
}

template <int W>
__global__ void __launch_bounds__(512, 1) search_kernel(const SearchArgs Ap) {
    extern __shared__ uint4 smem_raw[];
    uint32_t *sm = (uint32_t *)smem_raw;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    __shared__ int s_inst;
    __shared__ unsigned long long s_nodes, s_fails, s_sols;
    __shared__ SearchArgs A;
    if (threadIdx.x == 0) A = Ap;
    __syncthreads();
    const int per_warp = A.lsm * A.rmax + WS_WORDS;

    Worker<W> wk;
    wk.A = &A;
    wk.lsm = A.lsm;
    wk.slots = sm + A.stage_words + warp * per_warp;
    wk.ws = (WarpShared *)(wk.slots + A.lsm * A.rmax);
    wk.gw = blockIdx.x * A.warps + warp;
    wk.tick = 0;
    wk.init_shared();

    if (!A.batch) {
        const uint32_t *ib = stage_instance(A.arena + A.inst_off[0], sm, A.stage_words);
        __syncthreads();
        wk.I.load(ib);
        wk.S = wk.I.S;
        wk.R = record_words(wk.S, W);
        wk.T = A.teams;
        wk.run();
        wk.flush();
        return;
    }

    Team *T = A.teams + blockIdx.x;
    wk.T = T;
    for (;;) {
        if (threadIdx.x == 0) {
            s_inst = ld_volatile(&A.g->abort) ? A.n_inst : atomicAdd(&A.g->ticket, 1);
            s_nodes = 0;
            s_fails = 0;
            s_sols = 0;
        }
        __syncthreads();
        const int i = s_inst;
        if (i >= A.n_inst) break;
        const uint32_t *ib = stage_instance(A.arena + A.inst_off[i], sm, A.stage_words);
        __syncthreads();
        wk.I.load(ib);
        wk.S = wk.I.S;
        wk.R = record_words(wk.S, W);
        const unsigned long long n0 = wk.ws->nodes, f0 = wk.ws->fails, s0 = wk.ws->sols;
        if (lane == 0) wk.ws->sol_off = A.sol_off ? A.sol_off[i] : 0;
        __syncwarp();
        if (warp == 0) {
            if (lane == 0) {
                T->found = 0;
                T->work = 1;
                T->inst = i;
            }
            // root record: the instance's root domains, nothing to try yet, var = -1
            const uint32_t *root = A.arena + A.inst_off[i] + ib[H_OFF_ROOT];
            for (int k = lane; k < wk.R; k += 32)
                wk.slots[k] = k < wk.S ? root[k] : (k == wk.S + W ? 0xffffffffu : 0u);
            __syncwarp();
            __threadfence();
            q_push(A, T, wk.qseq(), wk.qrec(), wk.slots, wk.R, wk.S, W, false, 0u);
        }
        __syncthreads();
        wk.run();
        if (lane == 0) {
            atomicAdd(&s_nodes, wk.ws->nodes - n0);
            atomicAdd(&s_fails, wk.ws->fails - f0);
            atomicAdd(&s_sols, wk.ws->sols - s0);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            InstResult &r = A.results[i];
            const int st = ld_volatile(&A.g->status);
            r.status = T->found || s_sols > 0 ? 1 : (st != 0 ? st : 0);
            r.n = (int)ib[H_N];
            r.nodes = s_nodes;
            r.fails = s_fails;
            r.solutions = s_sols;
            r.sol_offset = A.sol_off ? A.sol_off[i] : 0;
        }
        __syncthreads();
    }
    wk.flush();
}

// ------------------------------------------------------------------ set-up kernels

// single-problem mode: team 0 holds the root record in slot 0 of its queue
__global__ void init_single_kernel(SearchArgs A) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int qcap = A.qmask + 1;
    for (int i = tid; i < qcap; i += gridDim.x * blockDim.x) A.qseq[i] = i == 0 ? 1u : (uint32_t)i;
    if (blockIdx.x == 0) {
        const uint32_t *ib = A.arena + A.inst_off[0];
        const int S = (int)ib[H_S], W = (int)ib[H_W];
        const int R = record_words(S, W);
        const uint32_t *root = ib + ib[H_OFF_ROOT];
        for (int k = threadIdx.x; k < R; k += blockDim.x)
            A.qrec[k] = k < S ? root[k] : (k == S + W ? 0xffffffffu : 0u);
        if (threadIdx.x == 0) {
            A.teams[0].work = 1;
            A.teams[0].tail = 1;
        }
    }
}

// batch mode: every team's queue starts empty
__global__ void init_batch_kernel(SearchArgs A, int teams) {
    const int qcap = A.qmask + 1;
    const long long total = (long long)teams * qcap;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        A.qseq[i] = (uint32_t)(i % qcap);
}

// ------------------------------------------------------------------ propagate kernel

template <int W>
__global__ void __launch_bounds__(256) propagate_kernel(PropArgs P) {
    extern __shared__ uint4 smem_raw[];
    uint32_t *sm = (uint32_t *)smem_raw;
    const uint32_t *ib = stage_instance(P.inst, sm, P.stage_words);
    __syncthreads();
    IV I;
    I.load(ib);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int warps = blockDim.x >> 5;
    const int per_warp = ((I.S + 3) & ~3) + 64;
    uint32_t *dom = sm + P.stage_words + warp * per_warp;
    uint32_t *chg = dom + ((I.S + 3) & ~3);
    uint32_t *evs = chg + 32;
    unsigned long long evals = 0;
    for (int s = blockIdx.x * warps + warp; s < P.count; s += gridDim.x * warps) {
        const uint32_t *src = P.din + (size_t)s * I.S;
        for (int k = lane; k < I.S; k += 32) dom[k] = src[k];
        __syncwarp();
        const bool failed = fixpoint<W>(I, dom, chg, evs, true, evals);
        __syncwarp();
        uint32_t *dst = P.dout + (size_t)s * I.S;
        for (int k = lane; k < I.S; k += 32) dst[k] = dom[k];
        if (lane == 0) P.failed[s] = failed ? 1 : 0;
        __syncwarp();
    }
}

// ------------------------------------------------------------------ host launchers

template <int W>
static cudaError_t launch_search_w(const SearchArgs &A, int blocks, int threads, size_t smem,
                                   cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(search_kernel<W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    search_kernel<W><<<blocks, threads, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_search(int W, const SearchArgs &A, int blocks, int threads, size_t smem,
                          cudaStream_t st) {
    switch (W) {
    case 1: return launch_search_w<1>(A, blocks, threads, smem, st);
    case 2: return launch_search_w<2>(A, blocks, threads, smem, st);
    case 4: return launch_search_w<4>(A, blocks, threads, smem, st);
    case 8: return launch_search_w<8>(A, blocks, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_search(int W, int threads, size_t smem, int *blocks_per_sm) {
    switch (W) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<1>, threads, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<2>, threads, smem);
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<4>, threads, smem);
    case 8: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<8>, threads, smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t set_search_smem(int W, size_t smem) {
    switch (W) {
    case 1: return cudaFuncSetAttribute(search_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 2: return cudaFuncSetAttribute(search_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 4: return cudaFuncSetAttribute(search_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 8: return cudaFuncSetAttribute(search_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_single(const SearchArgs &A, cudaStream_t st) {
    init_single_kernel<<<8, 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(const SearchArgs &A, int teams, cudaStream_t st) {
    init_batch_kernel<<<64, 256, 0, st>>>(A, teams);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_prop_w(const PropArgs &P, int blocks, int threads, size_t smem,
                                 cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(propagate_kernel<W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    propagate_kernel<W><<<blocks, threads, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_propagate(int W, const PropArgs &P, int blocks, int threads, size_t smem,
                             cudaStream_t st) {
    switch (W) {
    case 1: return launch_prop_w<1>(P, blocks, threads, smem, st);
    case 2: return launch_prop_w<2>(P, blocks, threads, smem, st);
    case 4: return launch_prop_w<4>(P, blocks, threads, smem, st);
    case 8: return launch_prop_w<8>(P, blocks, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace cubics
