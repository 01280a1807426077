// Device building blocks of the CUBICS search: domain helpers, the four propagators, the
// event-driven fixpoint and first-fail labeling.  One warp owns one search node at a time;
// its domains live in shared memory and every domain write is an atomicAnd, so bits are
// only ever cleared and concurrent lanes cannot re-add a removed value.
//
// Propagation (arxiv 1909.09213, Sections 1.1 and 2.2): every constraint whose scope
// changed is re-evaluated, the lanes of the warp working on constraints of one kind at a
// time, until a round changes no domain (the common fixpoint, which is unique because each
// propagator is monotone and contracting) or a domain becomes empty (failure).
//
// Shared memory is addressed through the block's dynamic array SM with 32-bit word
// offsets, so every access compiles to a shared-memory instruction.  The instance data is
// either staged at SM[0..) (STAGED) or read from global memory.
#pragma once
#include <stdint.h>
#include "internal.h"

namespace cubics {

#define FULLMASK 0xffffffffu

extern __shared__ __align__(16) uint32_t SM[];

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *(const volatile uint32_t *)p;
}
__device__ __forceinline__ int ld_volatile(const int32_t *p) {
    return *(const volatile int32_t *)p;
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// splitmix64 (Steele, Lea and Flood 2014): the output function applied to x + golden
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------------ domains (W words at SM[d])

template <int W>
__device__ __forceinline__ int dom_popc(int d) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) c += __popc(SM[d + k]);
    return c;
}

template <int W>
__device__ __forceinline__ int dom_min(int d) {   // lowest bit, -1 if empty
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const uint32_t w = SM[d + k];
        if (w) return (k << 5) + __ffs(w) - 1;
    }
    return -1;
}

template <int W>
__device__ __forceinline__ int dom_max(int d) {   // highest bit, -1 if empty
#pragma unroll
    for (int k = W - 1; k >= 0; --k) {
        const uint32_t w = SM[d + k];
        if (w) return (k << 5) + 31 - __clz(w);
    }
    return -1;
}

// bits of word k whose index is <= ub (ub may lie outside the window)
__device__ __forceinline__ uint32_t keep_le(int k, int ub) {
    const int lo = k << 5;
    if (ub < lo) return 0u;
    if (ub >= lo + 31) return FULLMASK;
    return FULLMASK >> (31 - (ub - lo));
}
// bits of word k whose index is >= lb
__device__ __forceinline__ uint32_t keep_ge(int k, int lb) {
    const int lo = k << 5;
    if (lb <= lo) return FULLMASK;
    if (lb > lo + 31) return 0u;
    return FULLMASK << (lb - lo);
}

__device__ __forceinline__ int floor_div(int q, int a) {
    int t = q / a;
    if ((q % a != 0) && ((q < 0) != (a < 0))) t -= 1;
    return t;
}
__device__ __forceinline__ int ceil_div(int q, int a) { return -floor_div(-q, a); }

// ------------------------------------------------------------------ instance view

template <bool ST>
struct IV {
    const uint32_t *g;   // instance block in global memory (read when not staged)
    int n, S, NW, lo0, flags;
    __device__ __forceinline__ uint32_t w(int i) const {
        if (ST) return SM[i];
        return __ldg(g + i);
    }
    __device__ __forceinline__ void load(const uint32_t *gp) {
        g = gp;
        n = (int)w(H_N);
        S = (int)w(H_S);
        NW = (int)w(H_NW);
        lo0 = (int)w(H_LO0);
        flags = (int)w(H_FLAGS);
    }
};

__device__ __forceinline__ void mark_changed(int chg, int v) {
    atomicOr(&SM[chg + (v >> 5)], 1u << (v & 31));
}

__device__ __forceinline__ bool ev_has(int evs, int v) {
    return (SM[evs + (v >> 5)] >> (v & 31)) & 1u;
}

// ------------------------------------------------------------------ propagators
// `dom` is the SM offset of the node's n*W domain words, `chg` of its changed-variable set.

// Binary table, both directions: D(x) keeps a iff row R[a] meets D(y); D(y) keeps b iff
// row C[b] meets D(x).  Lane l handles value l of each 32-value word.  Returns true on
// failure (a side became empty).
template <int W, bool ST>
__device__ bool revise_table(const IV<ST> &I, int dom, int chg, int t) {
    const int lane = lane_id();
    const int tb = (int)I.w(H_OFF_TAB) + 4 * t;
    const int x = (int)I.w(tb), y = (int)I.w(tb + 1);
    const int Rm = (int)I.w(tb + 2), Cm = (int)I.w(tb + 3);
    bool fail = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int p = side ? y : x, q = side ? x : y;
        const int M = side ? Cm : Rm;
        const int dp = dom + p * W, dq = dom + q * W;
        uint32_t dqw[W];
#pragma unroll
        for (int k = 0; k < W; ++k) dqw[k] = SM[dq + k];
        bool any = false, changed = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t dpw = SM[dp + w];
            bool keep = false;
            if ((dpw >> lane) & 1u) {
                const int row = M + ((w << 5) + lane) * W;
                uint32_t acc = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) acc |= I.w(row + k) & dqw[k];
                keep = acc != 0u;
            }
            const uint32_t nw = __ballot_sync(FULLMASK, keep);
            any |= nw != 0u;
            if (nw != dpw) {
                changed = true;
                if (lane == 0) atomicAnd(&SM[dp + w], nw);
            }
        }
        if (changed && lane == 0) mark_changed(chg, p);
        if (!any) fail = true;
        __syncwarp();
    }
    return fail;
}

// sum a_t x_t <= rhs, bounds reasoning: S = sum of each term's minimum; term t may not
// exceed rhs - (S - its minimum).  Lanes over terms.  Returns true on failure.
template <int W, bool ST>
__device__ bool revise_lin(const IV<ST> &I, int dom, int chg, int r) {
    const int lane = lane_id();
    const int row = (int)I.w(H_OFF_LIN_ROW) + 3 * r;
    const int t0 = (int)I.w(row), len = (int)I.w(row + 1), rhs = (int)I.w(row + 2);
    const int terms = (int)I.w(H_OFF_LIN_TERM) + 2 * t0;
    const int lo0 = I.lo0;
    int acc = 0;
    bool empty = false;
    for (int t = lane; t < len; t += 32) {
        const int a = (int)I.w(terms + 2 * t), v = (int)I.w(terms + 2 * t + 1);
        const int d = dom + v * W;
        const int mn = dom_min<W>(d);
        if (mn < 0) { empty = true; continue; }
        acc += a > 0 ? a * (lo0 + mn) : a * (lo0 + dom_max<W>(d));
    }
    if (__any_sync(FULLMASK, empty)) return true;
    const int S = __reduce_add_sync(FULLMASK, acc);
    if (S > rhs) return true;
    for (int t = lane; t < len; t += 32) {
        const int a = (int)I.w(terms + 2 * t), v = (int)I.w(terms + 2 * t + 1);
        const int d = dom + v * W;
        const int mn = dom_min<W>(d), mx = dom_max<W>(d);
        const int own = a > 0 ? a * (lo0 + mn) : a * (lo0 + mx);
        const int slack = rhs - (S - own);
        bool changed = false;
        if (a > 0) {
            const int ub = floor_div(slack, a) - lo0;       // keep bits <= ub
            if (ub < mx) {
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const uint32_t keep = keep_le(k, ub);
                    if (SM[d + k] & ~keep) { atomicAnd(&SM[d + k], keep); changed = true; }
                }
            }
        } else {
            const int lb = ceil_div(slack, a) - lo0;        // keep bits >= lb
            if (lb > mn) {
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const uint32_t keep = keep_ge(k, lb);
                    if (SM[d + k] & ~keep) { atomicAnd(&SM[d + k], keep); changed = true; }
                }
            }
        }
        if (changed) mark_changed(chg, v);
    }
    __syncwarp();
    return false;
}

// all different: values of fixed members leave the other members; failure when two
// members share a fixed value or the union of the domains is smaller than the group.
template <int W, bool ST>
__device__ bool revise_alldiff(const IV<ST> &I, int dom, int chg, int g) {
    const int lane = lane_id();
    const int grp = (int)I.w(H_OFF_AD_ROW) + 2 * g;
    const int m0 = (int)I.w(grp), len = (int)I.w(grp + 1);
    const int mem = (int)I.w(H_OFF_AD_MEM) + m0;
    uint32_t U1[W], UA[W];
#pragma unroll
    for (int k = 0; k < W; ++k) { U1[k] = 0; UA[k] = 0; }
    int nfix = 0;
    bool empty = false;
    for (int base = 0; base < len; base += 32) {
        const int j = base + lane;
        const bool act = j < len;
        const int v = act ? (int)I.w(mem + j) : 0;
        uint32_t d[W];
        int pc = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) { d[k] = act ? SM[dom + v * W + k] : 0u; pc += __popc(d[k]); }
        const bool fixed = act && pc == 1;
        empty |= act && pc == 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            U1[k] |= __reduce_or_sync(FULLMASK, fixed ? d[k] : 0u);
            UA[k] |= __reduce_or_sync(FULLMASK, d[k]);
        }
        nfix += __popc(__ballot_sync(FULLMASK, fixed));
    }
    if (__any_sync(FULLMASK, empty)) return true;
    int pu1 = 0, pua = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) { pu1 += __popc(U1[k]); pua += __popc(UA[k]); }
    if (nfix > pu1 || pua < len) return true;
    if (pu1 == 0) return false;
    bool fail = false;
    for (int base = 0; base < len; base += 32) {
        const int j = base + lane;
        if (j < len) {
            const int v = (int)I.w(mem + j);
            const int dv = dom + v * W;
            uint32_t d[W];
            int pc = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) { d[k] = SM[dv + k]; pc += __popc(d[k]); }
            const bool fixed = pc == 1;
            bool changed = false, any = false;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const uint32_t keep = fixed ? ~(U1[k] & ~d[k]) : ~U1[k];
                if (d[k] & ~keep) { atomicAnd(&SM[dv + k], keep); changed = true; }
                any |= (d[k] & keep) != 0u;
            }
            if (changed) mark_changed(chg, v);
            if (!any) fail = true;
        }
    }
    return __any_sync(FULLMASK, fail);
}

// all different, bounds-consistent (Section 4, second direction), by Hall intervals on the
// interval relaxation: when the members whose [min, max] lie inside an interval [a, b] are as
// many as its values, they use all of them, so no other member may keep a bound inside it
// (its min moves above b, its max below a; holes are kept, so a bound moves to the next value
// of the domain); more members than values fails.  Every Hall interval equals the interval
// from the least min to the greatest max of its members, so the candidates are the pairs
// (a member's min, a member's max).  Lane j holds member j (k <= ADB_MAX = 32); passes over
// the candidates repeat until one changes nothing.  Returns true on failure.  Out of line: only
// problems that post such groups run it, and inline its registers made every fixpoint spill.
template <int W, bool ST>
__device__ __noinline__ bool revise_alldiff_bc(const IV<ST> &I, int dom, int chg, int g) {
    const int lane = lane_id();
    const int grp = (int)I.w(H_OFF_ADB_ROW) + 2 * g;
    const int m0 = (int)I.w(grp), k = (int)I.w(grp + 1);
    const bool act = lane < k;
    const int v = act ? (int)I.w((int)I.w(H_OFF_ADB_MEM) + m0 + lane) : 0;
    const int dv = dom + v * W;
    int lo = act ? dom_min<W>(dv) : 0, hi = act ? dom_max<W>(dv) : 0;
    if (__any_sync(FULLMASK, act && lo < 0)) return true;
    bool mine_changed = false;
    for (bool again = true; again;) {
        again = false;
        for (int t = 0; t < k; ++t) {
            for (int u = 0; u < k; ++u) {
                const int a = __shfl_sync(FULLMASK, lo, t), b = __shfl_sync(FULLMASK, hi, u);
                if (b < a) continue;
                const uint32_t inside = __ballot_sync(FULLMASK, act && lo >= a && hi <= b);
                const int cnt = __popc(inside);
                if (cnt > b - a + 1) return true;
                if (cnt < b - a + 1) continue;
                bool moved = false;
                if (act && !((inside >> lane) & 1u) && ((lo >= a && lo <= b) || (hi >= a && hi <= b))) {
                    const bool cut_lo = lo >= a && lo <= b, cut_hi = hi >= a && hi <= b;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        uint32_t keep = FULLMASK;
                        if (cut_lo) keep &= keep_ge(w, b + 1);
                        if (cut_hi) keep &= keep_le(w, a - 1);
                        if (SM[dv + w] & ~keep) atomicAnd(&SM[dv + w], keep);
                    }
                    lo = dom_min<W>(dv);
                    hi = dom_max<W>(dv);
                    moved = true;
                    mine_changed = true;
                }
                if (__any_sync(FULLMASK, moved)) {
                    again = true;
                    if (__any_sync(FULLMASK, act && lo < 0)) {
                        if (mine_changed) mark_changed(chg, v);
                        return true;
                    }
                }
            }
        }
    }
    if (mine_changed) mark_changed(chg, v);
    __syncwarp();
    return false;
}

// Constraints of a kind whose scope meets the event set, from per-variable masks
// (mw words per variable at `mask`; bit c of word k = constraint 32k + c).  Calls f(c).
template <bool ST, typename F>
__device__ __forceinline__ bool for_scheduled(const IV<ST> &I, int evs, int mask, int mw, F f) {
    const int lane = lane_id();
    for (int wb = 0; wb < mw; wb += 8) {
        uint32_t acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0;
        for (int v = lane; v < I.n; v += 32) {
            if (!ev_has(evs, v)) continue;
            const int mv = mask + v * mw + wb;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (wb + k < mw) acc[k] |= I.w(mv + k);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (wb + k >= mw) break;
            uint32_t s = __reduce_or_sync(FULLMASK, acc[k]);
            while (s) {
                const int c = ((wb + k) << 5) + __ffs(s) - 1;
                s &= s - 1;
                if (f(c)) return true;
            }
        }
    }
    return false;
}

// ------------------------------------------------------------------ fixpoint

// The fixpoint of a problem with int_ne constraints only and one-word domains.  A newly fixed
// variable removes one value from each neighbour; a neighbour left with a single value is
// newly fixed in turn.  With one word per domain the atomicAnd's return value tells exactly
// which removal left one value (or none), so the next round's work is known without
// re-reading the domains.  SM[chg] holds the newly fixed variables (NW words); with full =
// true it is computed here from the domains.  Returns true when some domain became empty.
template <bool ST>
__device__ bool fixpoint_ne1(const IV<ST> &I, int dom, int chg, bool full, unsigned long long &evals,
                             unsigned long long &rounds) {
    const int lane = lane_id();
    const int n = I.n, NW = I.NW;
    if (full) {
        const int nun = (int)I.w(H_N_UN);
        const int un = (int)I.w(H_OFF_UN);
        for (int i = lane; i < nun; i += 32) {
            const uint32_t u = I.w(un + i);
            atomicAnd(&SM[dom + (int)(u & 0xffffu)], ~(1u << (u >> 16)));
        }
        __syncwarp();
        bool bad = false;
        for (int c = 0; c < NW; ++c) {
            const int v = (c << 5) + lane;
            const uint32_t d = v < n ? SM[dom + v] : 3u;
            bad |= d == 0u;
            const uint32_t f = __ballot_sync(FULLMASK, v < n && d != 0u && (d & (d - 1u)) == 0u);
            if (lane == 0) SM[chg + c] = f;
        }
        if (__any_sync(FULLMASK, bad)) return true;
        __syncwarp();
    }
    const int adj_start = (int)I.w(H_OFF_ADJ_START);
    const int adj = (int)I.w(H_OFF_ADJ);
    for (;;) {
        uint32_t fx = 0;
        if (lane < NW) {
            fx = SM[chg + lane];
            SM[chg + lane] = 0u;
        }
        if (!__any_sync(FULLMASK, fx != 0u)) return false;
        rounds++;
        __syncwarp();
        bool fail = false;
        for (int c = 0; c < NW; ++c) {
            uint32_t f = __shfl_sync(FULLMASK, fx, c);
            while (f) {
                const int v = (c << 5) + __ffs(f) - 1;
                f &= f - 1;
                evals++;
                const uint32_t dv = SM[dom + v];
                if (dv == 0u) { fail = true; continue; }   // its value was removed meanwhile
                const int val = __ffs(dv) - 1;
                const int e0 = (int)I.w(adj_start + v), e1 = (int)I.w(adj_start + v + 1);
                for (int e = e0 + lane; e < e1; e += 32) {
                    const uint32_t ent = I.w(adj + e);
                    const int t = (int)(ent & 0xffffu);
                    const int tb = val + (int)(int16_t)(ent >> 16);
                    if ((unsigned)tb < 32u) {
                        const uint32_t m = 1u << tb;
                        const uint32_t old = atomicAnd(&SM[dom + t], ~m);
                        if (old & m) {
                            const uint32_t nw = old & ~m;
                            if (nw == 0u) fail = true;
                            else if ((nw & (nw - 1u)) == 0u) atomicOr(&SM[chg + (t >> 5)], 1u << (t & 31));
                        }
                    }
                }
            }
        }
        if (__any_sync(FULLMASK, fail)) return true;
        __syncwarp();
    }
}

// ------------------------------------------------------------------ domains in registers
// One-word int_ne problems with at most 32 variables (FLAG_NE_REG): lane i of the warp holds
// D(x_i) in a register (lanes >= n hold 0 and take no part).  A fixed variable v with value
// bit a removes, from every D(x_i) at once, the bits a + off for the offsets off of the
// constraints between x_i and x_v: one 8-byte load of the offset mask M(v, i) per lane
// (consecutive words across the warp) and a funnel shift that aligns bit off + 31 with bit
// a + off.

// the offset mask of (fixed variable v, variable `lane`): staged or in global memory
template <bool ST>
__device__ __forceinline__ uint2 ne_mask(const IV<ST> &I, int nm, int v, int lane) {
    const int o = nm + 2 * ((v << 5) + lane);
    if (ST) return *reinterpret_cast<const uint2 *>(&SM[o]);
    return __ldg(reinterpret_cast<const uint2 *>(I.g + o));
}

// bits a + off (0 <= a <= 31) of the mask with bit off + 31 per offset: bit b of the result
// is mask bit b + 31 - a
__device__ __forceinline__ uint32_t ne_removed(uint2 m, int a) {
    return __funnelshift_r(m.x, m.y, 31 - a);
}

// Fixpoint of the node held in registers.  `pending` holds the fixed variables whose
// consequences have not been applied yet, `done` those whose consequences are already in the
// domains (the variables fixed in the parent, which is at its fixpoint: its domains contain
// the child's, so re-applying them would remove nothing).  Each round applies every pending
// variable's removals (their values are read at the start of the round: a pending variable
// is fixed, so its domain can only become empty, which fails the node anyway), then the
// variables newly left with one value become pending.  With x >= 0 the caller states that
// pending is {x}, just fixed to ax: the first round applies it without looking it up.
// Returns true when some domain became empty.
template <bool ST>
__device__ __forceinline__ bool fixpoint_reg(const IV<ST> &I, uint32_t &d, uint32_t pending,
                                             uint32_t done, unsigned long long &evals,
                                             unsigned long long &rounds, int x = -1,
                                             int ax = 0) {
    const int lane = lane_id();
    const bool act = lane < I.n;
    const int nm = (int)I.w(H_OFF_NEMASK);
    if (x >= 0) {             // pending = {x}, just fixed to ax: the first round applies it directly
        rounds++;
        evals++;
        d &= ~ne_removed(ne_mask(I, nm, x, lane), ax);
        done |= pending;
        if (__any_sync(FULLMASK, act && d == 0u)) return true;
        pending = __ballot_sync(FULLMASK, act && (d & (d - 1u)) == 0u) & ~done;
    }
    while (pending) {
        rounds++;
        evals += (unsigned)__popc(pending);
        const int a = __ffs(d) - 1;               // the value of each fixed variable
        uint32_t rm = 0;
        uint32_t p = pending;
        while (p) {                               // one fixed variable per step (a round mostly has one)
            const int v = __ffs(p) - 1;
            p &= p - 1;
            const int av = __shfl_sync(FULLMASK, a, v);
            rm |= ne_removed(ne_mask(I, nm, v, lane), av);
        }
        d &= ~rm;
        done |= pending;
        if (__any_sync(FULLMASK, act && d == 0u)) return true;
        pending = __ballot_sync(FULLMASK, act && (d & (d - 1u)) == 0u) & ~done;
    }
    return false;
}

// Fixpoints of two nodes at once, one per half-warp (n <= 16): lane 16h + i holds D(x_i) of
// node h.  The same rounds as fixpoint_reg for each half, in the same instructions: bits
// 16h + v of `pending` and `done` are node h's sets (a ballot yields both halves' sets in
// one word), a lane shuffles from its own half and loads the offset mask of its half's
// variable.  A half whose node failed stops at the round that emptied a domain, as
// fixpoint_reg returns there.  The nodes are siblings: in both, x was just fixed (to ax,
// the lane's node's value), so the first round applies x alone.  Returns the failed halves
// (0x0000ffff: node 0, 0xffff0000: node 1); evals and rounds of node h in bits
// 16h .. 16h + 15 of ev and rnd.
template <bool ST>
__device__ __forceinline__ uint32_t fixpoint_pair_reg(const IV<ST> &I, uint32_t &d, int x,
                                                      int ax, uint32_t done, uint32_t &ev,
                                                      uint32_t &rnd) {
    const int lane = lane_id();
    const int i = lane & 15;
    const uint32_t half = (lane & 16) ? 0xffff0000u : 0x0000ffffu;
    const bool act = i < I.n;
    const int nm = (int)I.w(H_OFF_NEMASK);
    const uint32_t done0 = done;
    uint32_t failed = 0u;
    // the first round: x alone is pending in both nodes, fixed to ax (the lane's node's value)
    uint32_t pending = (1u << x) | (1u << (16 + x));
    {
        rnd += 0x10001u;
        d &= ~ne_removed(ne_mask(I, nm, x, i), ax);
        done |= pending;
        const uint32_t empty = __ballot_sync(FULLMASK, act && d == 0u);
        failed = ((empty & 0xffffu) ? 0xffffu : 0u) | ((empty >> 16) ? 0xffff0000u : 0u);
        pending = __ballot_sync(FULLMASK, act && (d & (d - 1u)) == 0u) & ~done & ~failed;
    }
    while (pending) {
        rnd += ((pending & 0xffffu) ? 1u : 0u) | ((pending >> 16) ? 0x10000u : 0u);
        const int a = __ffs(d) - 1;               // the value of each fixed variable
        uint32_t rm = 0u;
        uint32_t p = pending & half;              // this lane's node (bit 16h + v)
        // one fixed variable of each node per step (a round mostly has one); a node with none
        // left takes a masked step on its own half's first lane
        while (__any_sync(FULLMASK, p != 0u)) {
            const bool has = p != 0u;
            const int v = has ? __ffs(p) - 1 : (lane & 16);
            p &= p - 1u;
            const int av = __shfl_sync(FULLMASK, a, v);
            const uint2 m = ne_mask(I, nm, v & 15, i);
            if (has) rm |= ne_removed(m, av);
        }
        d &= ~rm;
        done |= pending;
        const uint32_t empty = __ballot_sync(FULLMASK, act && d == 0u);
        failed |= ((empty & 0xffffu) ? 0xffffu : 0u) | ((empty >> 16) ? 0xffff0000u : 0u);
        pending = __ballot_sync(FULLMASK, act && (d & (d - 1u)) == 0u) & ~done & ~failed;
    }
    // each pending variable was applied once: the evaluations are the variables added to done
    const uint32_t added = done & ~done0;
    ev += (uint32_t)__popc(added & 0xffffu) | ((uint32_t)__popc(added >> 16) << 16);
    return failed;
}

// first-fail within each half-warp (n <= 16): the unfixed variable of the lane's node with the
// fewest values, lowest index on ties; -1 when every variable is fixed or `skip`
__device__ __forceinline__ int select_first_fail_pair(uint32_t d, int n, bool skip) {
    const int i = lane_id() & 15;
    uint32_t key = (!skip && i < n && (d & (d - 1u))) ? ((uint32_t)__popc(d) << 5) | (uint32_t)i
                                                       : 0xffffffffu;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(FULLMASK, key, o));
    return key == 0xffffffffu ? -1 : (int)(key & 31u);
}

// first-fail over register-held domains: the unfixed variable with the fewest values, lowest
// index on ties; -1 when every variable is fixed
__device__ __forceinline__ int select_first_fail_reg(uint32_t d, int n) {
    const int lane = lane_id();
    const uint32_t key = (lane < n && (d & (d - 1u))) ? ((uint32_t)__popc(d) << 5) | (uint32_t)lane
                                                       : 0xffffffffu;
    const uint32_t best = __reduce_min_sync(FULLMASK, key);
    return best == 0xffffffffu ? -1 : (int)(best & 31u);
}

// Propagates the node at SM[dom] (S words) to its fixpoint.  SM[chg] (NW words) holds the
// variables changed since the last fixpoint; with full = true every variable counts as
// changed and unary constraints are applied first.  SM[evs] is NW words of scratch.
// Returns true when some domain became empty.
template <int W, bool ST>
__device__ bool fixpoint(const IV<ST> &I, int dom, int chg, int evs, bool full,
                         unsigned long long &evals, unsigned long long &rounds, int list = -1) {
    const int lane = lane_id();
    const int n = I.n, NW = I.NW;
    if (I.flags & FLAG_TRIVIAL_FAIL) return true;
    if (W == 1 && (I.flags & FLAG_NE_ONLY)) return fixpoint_ne1<ST>(I, dom, chg, full, evals, rounds);
    if (full) {
        if (lane < NW) {
            const int rem = n - (lane << 5);
            SM[chg + lane] = rem >= 32 ? FULLMASK : ((1u << rem) - 1u);
        }
        const int nun = (int)I.w(H_N_UN);
        const int un = (int)I.w(H_OFF_UN);
        for (int i = lane; i < nun; i += 32) {
            const uint32_t u = I.w(un + i);
            const int x = (int)(u & 0xffffu), bit = (int)(u >> 16);
            atomicAnd(&SM[dom + x * W + (bit >> 5)], ~(1u << (bit & 31)));
        }
        __syncwarp();
    }
    const int adj_start = (int)I.w(H_OFF_ADJ_START);
    const int adj = (int)I.w(H_OFF_ADJ);
    const int n_tab = (int)I.w(H_N_TAB);
    const int n_lin = (int)I.w(H_N_LIN), n_ad = (int)I.w(H_N_AD), n_adb = (int)I.w(H_N_ADB);
    const bool has_ne = I.w(H_N_NE) != 0u;
    for (;;) {
        // 1. this round's events: the variables changed in the previous round
        uint32_t ev = 0;
        if (lane < NW) {
            ev = SM[chg + lane];
            SM[evs + lane] = ev;
            SM[chg + lane] = 0;
        }
        if (!__any_sync(FULLMASK, ev != 0u)) return false;
        rounds++;
        __syncwarp();
        // 2. empty and fixed variables among them
        uint32_t fxw = 0;
        bool bad = false;
        for (int c = 0; c < NW; ++c) {
            const uint32_t e = SM[evs + c];
            if (!e) continue;
            const int v = (c << 5) + lane;
            const bool mine = (e >> lane) & 1u;
            const int pc = mine ? dom_popc<W>(dom + v * W) : 2;
            bad |= pc == 0;
            const uint32_t f = __ballot_sync(FULLMASK, mine && pc == 1);
            if (lane == c) fxw = f;
        }
        if (__any_sync(FULLMASK, bad)) return true;
        // 3. int_ne: a newly fixed variable forbids one value of each neighbour
        bool fail = false;
        if (has_ne) {
            for (int c = 0; c < NW; ++c) {
                uint32_t f = __shfl_sync(FULLMASK, fxw, c);
                while (f) {
                    const int v = (c << 5) + __ffs(f) - 1;
                    f &= f - 1;
                    const int val = __shfl_sync(FULLMASK, dom_min<W>(dom + v * W), 0);
                    if (val < 0) continue;                  // emptied this round: caught next
                    const int e0 = (int)I.w(adj_start + v), e1 = (int)I.w(adj_start + v + 1);
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const uint32_t ent = I.w(adj + e);
                        const int t = (int)(ent & 0xffffu);
                        const int tb = val + (int)(int16_t)(ent >> 16);
                        if ((unsigned)tb < (unsigned)(32 * W)) {
                            const uint32_t m = 1u << (tb & 31);
                            const uint32_t old = atomicAnd(&SM[dom + t * W + (tb >> 5)], ~m);
                            if (old & m) {
                                mark_changed(chg, t);
                                if (W == 1 && (old & ~m) == 0u) fail = true;
                            }
                        }
                    }
                    if (lane == 0) evals++;
                }
            }
            if (__any_sync(FULLMASK, fail)) return true;
        }
        // 4. tables whose x or y changed
        if (n_tab && W == 1 && list >= 0) {
            // One lane per table, over a compacted list of the scheduled tables, so every lane
            // has a table.  D(x) keeps the values in the union of the columns C[b], b in D(y)
            // (revised when D(y) changed); D(y) those in the union of the rows R[a], a in D(x)
            // (revised when D(x) changed or was just revised).  A union stops growing once
            // it covers the domain it filters.
            const int tab = (int)I.w(H_OFF_TAB);
            int cnt = 0;
            for (int base = 0; base < n_tab; base += 32) {
                const int t = base + lane;
                uint32_t fl = 0;
                if (t < n_tab) {
                    fl = (ev_has(evs, (int)I.w(tab + 4 * t)) ? 1u : 0u) |
                         (ev_has(evs, (int)I.w(tab + 4 * t + 1)) ? 2u : 0u);
                }
                const uint32_t mk = __ballot_sync(FULLMASK, fl != 0u);
                if (fl) SM[list + cnt + __popc(mk & ((1u << lane) - 1u))] = (uint32_t)t | (fl << 30);
                cnt += __popc(mk);
            }
            __syncwarp();
            if (lane == 0) evals += cnt;
            for (int i0 = 0; i0 < cnt; i0 += 32) {
                const int i = i0 + lane;
                if (i < cnt) {
                    const uint32_t e = SM[list + i];
                    const int te = tab + 4 * (int)(e & 0x3fffffffu);
                    uint32_t fl = e >> 30;
                    const int x = (int)I.w(te), y = (int)I.w(te + 1);
                    uint32_t dx = SM[dom + x];
                    const uint32_t dy = SM[dom + y];
                    if (fl & 2u) {
                        const int Cm = (int)I.w(te + 3);
                        uint32_t acc = 0;
                        for (uint32_t m = dy; m && (acc & dx) != dx; m &= m - 1) acc |= I.w(Cm + __ffs(m) - 1);
                        const uint32_t kx = dx & acc;
                        if (kx != dx) {
                            const uint32_t old = atomicAnd(&SM[dom + x], kx);
                            if (old & ~kx) mark_changed(chg, x);
                            if ((old & kx) == 0u) fail = true;
                            fl |= 1u;
                            dx = kx;
                        }
                    }
                    if ((fl & 1u) && dx) {
                        const int Rm = (int)I.w(te + 2);
                        uint32_t acc = 0;
                        for (uint32_t m = dx; m && (acc & dy) != dy; m &= m - 1) acc |= I.w(Rm + __ffs(m) - 1);
                        const uint32_t ky = dy & acc;
                        if (ky != dy) {
                            const uint32_t old = atomicAnd(&SM[dom + y], ky);
                            if (old & ~ky) mark_changed(chg, y);
                            if ((old & ky) == 0u) fail = true;
                        }
                    }
                }
            }
            if (__any_sync(FULLMASK, fail)) return true;
        } else if (n_tab) {
            const int tab = (int)I.w(H_OFF_TAB);
            for (int base = 0; base < n_tab; base += 32) {
                const int t = base + lane;
                bool ex = false, ey = false;
                int x = 0, y = 0;
                if (t < n_tab) {
                    x = (int)I.w(tab + 4 * t);
                    y = (int)I.w(tab + 4 * t + 1);
                    ex = ev_has(evs, x);
                    ey = ev_has(evs, y);
                }
                if (W == 1) {
                    // Lanes over the 32 values.  The supported values of x are the union of the
                    // columns C[b] over b in D(y), those of y the union of the rows R[a] over
                    // a in D(x): one coalesced load and one OR-reduction per side.  D(x) is
                    // revised when D(y) changed, D(y) when D(x) changed or was just revised.
                    // TG scheduled tables go through together as independent chains.
                    constexpr int TG = 4;
                    const uint32_t flags = (ex ? 1u : 0u) | (ey ? 2u : 0u);
                    uint32_t sm = __ballot_sync(FULLMASK, flags != 0u);
                    if (lane == 0) evals += __popc(sm);
                    while (sm) {
                        int tx[TG], ty[TG], Rm[TG], Cm[TG];
                        uint32_t fl[TG], dx[TG], dy[TG], c[TG];
#pragma unroll
                        for (int g = 0; g < TG; ++g) {
                            const int src = sm ? __ffs(sm) - 1 : 0;
                            fl[g] = sm ? __shfl_sync(FULLMASK, flags, src) : 0u;
                            sm &= sm - 1;
                            tx[g] = __shfl_sync(FULLMASK, x, src);
                            ty[g] = __shfl_sync(FULLMASK, y, src);
                            const int e = tab + 4 * (base + src);
                            Rm[g] = (int)I.w(e + 2);
                            Cm[g] = (int)I.w(e + 3);
                        }
                        // x sides (tables whose y changed)
#pragma unroll
                        for (int g = 0; g < TG; ++g) {
                            dx[g] = SM[dom + tx[g]];
                            dy[g] = SM[dom + ty[g]];
                            c[g] = ((fl[g] & 2u) && ((dy[g] >> lane) & 1u)) ? I.w(Cm[g] + lane) : 0u;
                        }
#pragma unroll
                        for (int g = 0; g < TG; ++g) c[g] = __reduce_or_sync(FULLMASK, c[g]);
#pragma unroll
                        for (int g = 0; g < TG; ++g) {
                            if (fl[g] & 2u) {
                                const uint32_t kx = dx[g] & c[g];
                                if (kx != dx[g]) {
                                    if (lane == g) {
                                        const uint32_t old = atomicAnd(&SM[dom + tx[g]], kx);
                                        if (old & ~kx) mark_changed(chg, tx[g]);
                                        if ((old & kx) == 0u) fail = true;
                                    }
                                    fl[g] |= 1u;          // D(x) shrank: revise D(y) too
                                    dx[g] = kx;
                                }
                            }
                        }
                        // y sides (tables whose x changed or was just revised)
#pragma unroll
                        for (int g = 0; g < TG; ++g)
                            c[g] = ((fl[g] & 1u) && ((dx[g] >> lane) & 1u)) ? I.w(Rm[g] + lane) : 0u;
#pragma unroll
                        for (int g = 0; g < TG; ++g) c[g] = __reduce_or_sync(FULLMASK, c[g]);
#pragma unroll
                        for (int g = 0; g < TG; ++g) {
                            if (fl[g] & 1u) {
                                const uint32_t ky = dy[g] & c[g];
                                if (ky != dy[g] && lane == g) {
                                    const uint32_t old = atomicAnd(&SM[dom + ty[g]], ky);
                                    if (old & ~ky) mark_changed(chg, ty[g]);
                                    if ((old & ky) == 0u) fail = true;
                                }
                            }
                        }
                        __syncwarp();
                    }
                } else {
                    uint32_t sm = __ballot_sync(FULLMASK, ex || ey);
                    while (sm) {
                        const int tt = base + __ffs(sm) - 1;
                        sm &= sm - 1;
                        if (lane == 0) evals++;
                        if (revise_table<W, ST>(I, dom, chg, tt)) return true;
                    }
                }
            }
            if (__any_sync(FULLMASK, fail)) return true;
        }
        // 5. linear rows and 6. alldifferent groups whose scope changed (value elimination)
        if (n_lin) {
            if (for_scheduled<ST>(I, evs, (int)I.w(H_OFF_LIN_MASK), (int)I.w(H_LIN_MW), [&](int r) {
                    if (lane == 0) evals++;
                    return revise_lin<W, ST>(I, dom, chg, r);
                }))
                return true;
        }
        if (n_ad) {
            if (for_scheduled<ST>(I, evs, (int)I.w(H_OFF_AD_MASK), (int)I.w(H_AD_MW), [&](int g) {
                    if (lane == 0) evals++;
                    return revise_alldiff<W, ST>(I, dom, chg, g);
                }))
                return true;
        }
        // 7. bounds-consistent alldifferent groups whose scope changed
        if (n_adb) {
            if (for_scheduled<ST>(I, evs, (int)I.w(H_OFF_ADB_MASK), (int)I.w(H_ADB_MW), [&](int g) {
                    if (lane == 0) evals++;
                    return revise_alldiff_bc<W, ST>(I, dom, chg, g);
                }))
                return true;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ one node, many warps
// The fixpoint of one node computed by every warp of the block (constraint-parallel
// propagation of a node too large for one warp: the constraints of each kind are grouped,
// as Section 2.2 groups them, and shared out among the warps): in each round every warp reads
// the same event set and takes its share of the work of each kind (the fixed variables of
// int_ne by index, the 32-table chunks of one-word tables, rows, groups and multi-word tables
// by index); domain writes stay atomicAnd, so concurrent warps only ever clear bits; a block
// barrier ends the round.  Every thread of the block calls it.  Returns true (in every
// thread) when some domain became empty.
template <int W, bool ST>
__device__ bool fixpoint_block(const IV<ST> &I, int dom, int chg, int evs, bool full,
                               unsigned long long &evals, unsigned long long &rounds) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int n = I.n, NW = I.NW;
    if (I.flags & FLAG_TRIVIAL_FAIL) return true;
    if (full) {
        for (int c = threadIdx.x; c < NW; c += blockDim.x) {
            const int rem = n - (c << 5);
            SM[chg + c] = rem >= 32 ? FULLMASK : ((1u << rem) - 1u);
        }
        const int nun = (int)I.w(H_N_UN), un = (int)I.w(H_OFF_UN);
        for (int i = threadIdx.x; i < nun; i += blockDim.x) {
            const uint32_t u = I.w(un + i);
            const int x = (int)(u & 0xffffu), bit = (int)(u >> 16);
            atomicAnd(&SM[dom + x * W + (bit >> 5)], ~(1u << (bit & 31)));
        }
    }
    __syncthreads();
    const int adj_start = (int)I.w(H_OFF_ADJ_START), adj = (int)I.w(H_OFF_ADJ);
    const int n_tab = (int)I.w(H_N_TAB);
    const int n_lin = (int)I.w(H_N_LIN), n_ad = (int)I.w(H_N_AD), n_adb = (int)I.w(H_N_ADB);
    const bool has_ne = I.w(H_N_NE) != 0u;
    for (;;) {
        // 1. this round's events (every thread reads them after the barrier)
        for (int c = threadIdx.x; c < NW; c += blockDim.x) {
            SM[evs + c] = SM[chg + c];
            SM[chg + c] = 0u;
        }
        __syncthreads();
        bool any_ev = false;
        for (int c = 0; c < NW; ++c) any_ev |= SM[evs + c] != 0u;
        if (!any_ev) return false;
        rounds++;
        // 2. empty and fixed variables among the events (each warp computes the fixed set)
        uint32_t fxw = 0;
        bool fail = false;
        for (int c = 0; c < NW; ++c) {
            const uint32_t e = SM[evs + c];
            if (!e) continue;
            const int v = (c << 5) + lane;
            const bool mine = (e >> lane) & 1u;
            const int pc = mine ? dom_popc<W>(dom + v * W) : 2;
            fail |= pc == 0;
            const uint32_t f = __ballot_sync(FULLMASK, mine && pc == 1);
            if (lane == c) fxw = f;
        }
        // 3. int_ne: the fixed variables v with v mod nwarps == warp
        if (has_ne && !__any_sync(FULLMASK, fail)) {
            for (int c = 0; c < NW; ++c) {
                uint32_t f = __shfl_sync(FULLMASK, fxw, c);
                while (f) {
                    const int v = (c << 5) + __ffs(f) - 1;
                    f &= f - 1;
                    if (v % nwarps != warp) continue;
                    const int val = __shfl_sync(FULLMASK, dom_min<W>(dom + v * W), 0);
                    if (val < 0) continue;                  // emptied this round: caught next
                    const int e0 = (int)I.w(adj_start + v), e1 = (int)I.w(adj_start + v + 1);
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const uint32_t ent = I.w(adj + e);
                        const int t = (int)(ent & 0xffffu);
                        const int tb = val + (int)(int16_t)(ent >> 16);
                        if ((unsigned)tb < (unsigned)(32 * W)) {
                            const uint32_t m = 1u << (tb & 31);
                            const uint32_t old = atomicAnd(&SM[dom + t * W + (tb >> 5)], ~m);
                            if (old & m) mark_changed(chg, t);
                        }
                    }
                    if (lane == 0) evals++;
                }
            }
        }
        // 4. tables whose x or y changed: 32-table chunks (one word) or tables (wider) by warp
        if (n_tab && !__any_sync(FULLMASK, fail)) {
            const int tab = (int)I.w(H_OFF_TAB);
            for (int base = 0; base < n_tab && !fail; base += 32) {
                const int t = base + lane;
                bool ex = false, ey = false;
                if (t < n_tab) {
                    ex = ev_has(evs, (int)I.w(tab + 4 * t));
                    ey = ev_has(evs, (int)I.w(tab + 4 * t + 1));
                }
                uint32_t sm = __ballot_sync(FULLMASK, ex || ey);
                while (sm) {
                    const int tt = base + __ffs(sm) - 1;
                    sm &= sm - 1;
                    if (tt % nwarps != warp) continue;
                    if (lane == 0) evals++;
                    if (revise_table<W, ST>(I, dom, chg, tt)) {
                        fail = true;
                        break;
                    }
                }
            }
        }
        // 5. rows, 6. value-elimination groups, 7. bounds-consistent groups, by index
        if (n_lin && !__any_sync(FULLMASK, fail)) {
            fail = for_scheduled<ST>(I, evs, (int)I.w(H_OFF_LIN_MASK), (int)I.w(H_LIN_MW), [&](int r) {
                if (r % nwarps != warp) return false;
                if (lane == 0) evals++;
                return revise_lin<W, ST>(I, dom, chg, r);
            });
        }
        if (n_ad && !__any_sync(FULLMASK, fail)) {
            fail = for_scheduled<ST>(I, evs, (int)I.w(H_OFF_AD_MASK), (int)I.w(H_AD_MW), [&](int g) {
                if (g % nwarps != warp) return false;
                if (lane == 0) evals++;
                return revise_alldiff<W, ST>(I, dom, chg, g);
            });
        }
        if (n_adb && !__any_sync(FULLMASK, fail)) {
            fail = for_scheduled<ST>(I, evs, (int)I.w(H_OFF_ADB_MASK), (int)I.w(H_ADB_MW), [&](int g) {
                if (g % nwarps != warp) return false;
                if (lane == 0) evals++;
                return revise_alldiff_bc<W, ST>(I, dom, chg, g);
            });
        }
        fail = __any_sync(FULLMASK, fail);
        if (__syncthreads_or(fail ? 1 : 0)) return true;
    }
}

// First-fail: the unfixed variable with the fewest values, lowest index on ties; -1 when
// every variable is fixed.
template <int W>
__device__ __forceinline__ int select_first_fail(int dom, int n) {
    unsigned best = 0xffffffffu;
    for (int v = lane_id(); v < n; v += 32) {
        const int pc = dom_popc<W>(dom + v * W);
        if (pc > 1) best = min(best, ((unsigned)pc << 16) | (unsigned)v);
    }
    best = __reduce_min_sync(FULLMASK, best);
    return best == 0xffffffffu ? -1 : (int)(best & 0xffffu);
}

// ------------------------------------------------------------------ copies (words % 4 == 0)

// shared -> shared
__device__ __forceinline__ void copy_ss(int dst, int src, int words) {
    uint4 *S4 = reinterpret_cast<uint4 *>(SM);
    for (int i = lane_id(); i < (words >> 2); i += 32) S4[(dst >> 2) + i] = S4[(src >> 2) + i];
}
// shared -> global
__device__ __forceinline__ void copy_sg(uint32_t *dst, int src, int words) {
    const uint4 *S4 = reinterpret_cast<const uint4 *>(SM);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = lane_id(); i < (words >> 2); i += 32) d[i] = S4[(src >> 2) + i];
}
// global -> shared (cg: records written by other SMs)
__device__ __forceinline__ void copy_gs_cg(int dst, const uint32_t *src, int words) {
    uint4 *S4 = reinterpret_cast<uint4 *>(SM);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int i = lane_id(); i < (words >> 2); i += 32) S4[(dst >> 2) + i] = __ldcg(s + i);
}
// global -> global
__device__ __forceinline__ void copy_gg(uint32_t *dst, const uint32_t *src, int words) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int i = lane_id(); i < (words >> 2); i += 32) d[i] = s[i];
}

}  // namespace cubics
