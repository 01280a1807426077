// Device building blocks of the CUBICS search: domain helpers, the four propagators, the
// event-driven fixpoint and first-fail labeling.  One warp owns one search node at a time;
// its domains live in shared memory and every domain write is an atomicAnd, so bits are
// only ever cleared and concurrent lanes cannot re-add a removed value.
//
// Propagation (arxiv 1909.09213, Sections 1.1 and 2.2): every constraint whose scope
// changed is re-evaluated, all lanes of the warp working on constraints of one kind at a
// time, until a round changes no domain (the common fixpoint, which is unique because each
// propagator is monotone and contracting) or a domain becomes empty (failure).
#pragma once
#include <stdint.h>
#include "internal.h"

namespace cubics {

#define FULLMASK 0xffffffffu

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *(const volatile uint32_t *)p;
}
__device__ __forceinline__ int ld_volatile(const int32_t *p) {
    return *(const volatile int32_t *)p;
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

// ------------------------------------------------------------------ domains (W words)

template <int W>
__device__ __forceinline__ int dom_popc(const uint32_t *d) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) c += __popc(d[k]);
    return c;
}

template <int W>
__device__ __forceinline__ int dom_min(const uint32_t *d) {   // lowest bit, -1 if empty
#pragma unroll
    for (int k = 0; k < W; ++k) {
        uint32_t w = d[k];
        if (w) return (k << 5) + __ffs(w) - 1;
    }
    return -1;
}

template <int W>
__device__ __forceinline__ int dom_max(const uint32_t *d) {   // highest bit, -1 if empty
#pragma unroll
    for (int k = W - 1; k >= 0; --k) {
        uint32_t w = d[k];
        if (w) return (k << 5) + 31 - __clz(w);
    }
    return -1;
}

// bits of word k whose index is <= ub (ub may lie outside the window)
__device__ __forceinline__ uint32_t keep_le(int k, int ub) {
    int lo = k << 5;
    if (ub < lo) return 0u;
    if (ub >= lo + 31) return FULLMASK;
    return FULLMASK >> (31 - (ub - lo));
}
// bits of word k whose index is >= lb
__device__ __forceinline__ uint32_t keep_ge(int k, int lb) {
    int lo = k << 5;
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

struct IV {
    const uint32_t *b;   // instance block: shared memory when staged, else global
    int n, S, NW, lo0, flags;
    __device__ __forceinline__ void load(const uint32_t *p) {
        b = p;
        n = (int)p[H_N];
        S = (int)p[H_S];
        NW = (int)p[H_NW];
        lo0 = (int)p[H_LO0];
        flags = (int)p[H_FLAGS];
    }
    __device__ __forceinline__ uint32_t h(int i) const { return b[i]; }
};

__device__ __forceinline__ void mark_changed(uint32_t *chg, int v) {
    atomicOr(&chg[v >> 5], 1u << (v & 31));
}

__device__ __forceinline__ bool ev_has(const uint32_t *evs, int v) {
    return (evs[v >> 5] >> (v & 31)) & 1u;
}

// ------------------------------------------------------------------ propagators

// Binary table, both directions: D(x) keeps a iff row R[a] meets D(y); D(y) keeps b iff
// row C[b] meets D(x).  Lane l handles value l of each 32-value word.  Returns true on
// failure (a side became empty).
template <int W>
__device__ bool revise_table(const IV &I, uint32_t *dom, uint32_t *chg, int t) {
    const int lane = lane_id();
    const uint32_t *tb = I.b + I.h(H_OFF_TAB) + 4 * t;
    const int x = (int)tb[0], y = (int)tb[1];
    const uint32_t *Rm = I.b + tb[2];
    const uint32_t *Cm = I.b + tb[3];
    bool fail = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int p = side ? y : x, q = side ? x : y;
        const uint32_t *M = side ? Cm : Rm;
        uint32_t *dp = dom + p * W;
        const uint32_t *dq = dom + q * W;
        uint32_t dqw[W];
#pragma unroll
        for (int k = 0; k < W; ++k) dqw[k] = dq[k];
        bool any = false, changed = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t dpw = dp[w];
            bool keep = false;
            if ((dpw >> lane) & 1u) {
                const uint32_t *row = M + ((w << 5) + lane) * W;
                uint32_t acc = 0;
#pragma unroll
                for (int k = 0; k < W; ++k) acc |= row[k] & dqw[k];
                keep = acc != 0u;
            }
            const uint32_t nw = __ballot_sync(FULLMASK, keep);
            any |= nw != 0u;
            if (nw != dpw) {
                changed = true;
                if (lane == 0) atomicAnd(&dp[w], nw);
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
template <int W>
__device__ bool revise_lin(const IV &I, uint32_t *dom, uint32_t *chg, int r) {
    const int lane = lane_id();
    const uint32_t *row = I.b + I.h(H_OFF_LIN_ROW) + 3 * r;
    const int t0 = (int)row[0], len = (int)row[1], rhs = (int)row[2];
    const int *terms = (const int *)(I.b + I.h(H_OFF_LIN_TERM)) + 2 * t0;
    const int lo0 = I.lo0;
    int acc = 0;
    bool empty = false;
    for (int t = lane; t < len; t += 32) {
        const int a = terms[2 * t], v = terms[2 * t + 1];
        const uint32_t *d = dom + v * W;
        const int mn = dom_min<W>(d);
        if (mn < 0) { empty = true; continue; }
        acc += a > 0 ? a * (lo0 + mn) : a * (lo0 + dom_max<W>(d));
    }
    if (__any_sync(FULLMASK, empty)) return true;
    const int S = __reduce_add_sync(FULLMASK, acc);
    if (S > rhs) return true;
    for (int t = lane; t < len; t += 32) {
        const int a = terms[2 * t], v = terms[2 * t + 1];
        uint32_t *d = dom + v * W;
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
                    if (d[k] & ~keep) { atomicAnd(&d[k], keep); changed = true; }
                }
            }
        } else {
            const int lb = ceil_div(slack, a) - lo0;        // keep bits >= lb
            if (lb > mn) {
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const uint32_t keep = keep_ge(k, lb);
                    if (d[k] & ~keep) { atomicAnd(&d[k], keep); changed = true; }
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
template <int W>
__device__ bool revise_alldiff(const IV &I, uint32_t *dom, uint32_t *chg, int g) {
    const int lane = lane_id();
    const uint32_t *grp = I.b + I.h(H_OFF_AD_ROW) + 2 * g;
    const int m0 = (int)grp[0], len = (int)grp[1];
    const uint32_t *mem = I.b + I.h(H_OFF_AD_MEM) + m0;
    uint32_t U1[W], UA[W];
#pragma unroll
    for (int k = 0; k < W; ++k) { U1[k] = 0; UA[k] = 0; }
    int nfix = 0;
    bool empty = false;
    for (int base = 0; base < len; base += 32) {
        const int j = base + lane;
        const bool act = j < len;
        const int v = act ? (int)mem[j] : 0;
        uint32_t d[W];
        int pc = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) { d[k] = act ? dom[v * W + k] : 0u; pc += __popc(d[k]); }
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
            const int v = (int)mem[j];
            uint32_t *dv = dom + v * W;
            uint32_t d[W];
            int pc = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) { d[k] = dv[k]; pc += __popc(d[k]); }
            const bool fixed = pc == 1;
            bool changed = false, any = false;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const uint32_t keep = fixed ? ~(U1[k] & ~d[k]) : ~U1[k];
                if (d[k] & ~keep) { atomicAnd(&dv[k], keep); changed = true; }
                any |= (d[k] & keep) != 0u;
            }
            if (changed) mark_changed(chg, v);
            if (!any) fail = true;
        }
    }
    return __any_sync(FULLMASK, fail);
}

// Constraints of a kind whose scope meets the event set, from per-variable masks
// (mw words per variable; bit c of word k = constraint 32k + c).  Calls f(c) for each.
template <typename F>
__device__ __forceinline__ bool for_scheduled(const IV &I, const uint32_t *evs, const uint32_t *mask,
                                              int mw, F f) {
    const int lane = lane_id();
    for (int wb = 0; wb < mw; wb += 8) {
        uint32_t acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0;
        for (int v = lane; v < I.n; v += 32) {
            if (!ev_has(evs, v)) continue;
            const uint32_t *mv = mask + v * mw + wb;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (wb + k < mw) acc[k] |= mv[k];
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

// Propagates `dom` (S words in shared memory) to the fixpoint.  `chg` (NW words, shared)
// holds the variables changed since the last fixpoint; with full = true every variable
// counts as changed and unary constraints are applied first.  `evs` is NW words of shared
// scratch.  Returns true when some domain became empty.
template <int W>
__device__ bool fixpoint(const IV &I, uint32_t *dom, uint32_t *chg, uint32_t *evs, bool full,
                         unsigned long long &evals) {
    const int lane = lane_id();
    const int n = I.n, NW = I.NW;
    if (I.flags & FLAG_TRIVIAL_FAIL) return true;
    if (full) {
        if (lane < NW) {
            const int rem = n - (lane << 5);
            chg[lane] = rem >= 32 ? FULLMASK : ((1u << rem) - 1u);
        }
        const int nun = (int)I.h(H_N_UN);
        const uint32_t *un = I.b + I.h(H_OFF_UN);
        for (int i = lane; i < nun; i += 32) {
            const uint32_t u = un[i];
            const int x = (int)(u & 0xffffu), bit = (int)(u >> 16);
            atomicAnd(&dom[x * W + (bit >> 5)], ~(1u << (bit & 31)));
        }
        __syncwarp();
    }
    const uint32_t *adj_start = I.b + I.h(H_OFF_ADJ_START);
    const uint32_t *adj = I.b + I.h(H_OFF_ADJ);
    const int n_tab = (int)I.h(H_N_TAB);
    const int n_lin = (int)I.h(H_N_LIN), n_ad = (int)I.h(H_N_AD);
    const bool has_ne = I.h(H_N_NE) != 0;
    for (;;) {
        // 1. this round's events: the variables changed in the previous round
        uint32_t ev = 0;
        if (lane < NW) {
            ev = chg[lane];
            evs[lane] = ev;
            chg[lane] = 0;
        }
        if (!__any_sync(FULLMASK, ev != 0u)) return false;
        __syncwarp();
        // 2. empty and fixed variables among them
        uint32_t fxw = 0;
        bool bad = false;
        for (int c = 0; c < NW; ++c) {
            const uint32_t e = evs[c];
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
                    const int e0 = (int)adj_start[v], e1 = (int)adj_start[v + 1];
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const uint32_t ent = adj[e];
                        const int t = (int)(ent & 0xffffu);
                        const int tb = val + (int)(int16_t)(ent >> 16);
                        if ((unsigned)tb < (unsigned)(32 * W)) {
                            const uint32_t m = 1u << (tb & 31);
                            const uint32_t old = atomicAnd(&dom[t * W + (tb >> 5)], ~m);
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
        for (int base = 0; base < n_tab; base += 32) {
            const int t = base + lane;
            bool s = false;
            if (t < n_tab) {
                const uint32_t *tb = I.b + I.h(H_OFF_TAB) + 4 * t;
                s = ev_has(evs, (int)tb[0]) || ev_has(evs, (int)tb[1]);
            }
            uint32_t sm = __ballot_sync(FULLMASK, s);
            while (sm) {
                const int tt = base + __ffs(sm) - 1;
                sm &= sm - 1;
                if (lane == 0) evals++;
                if (revise_table<W>(I, dom, chg, tt)) return true;
            }
        }
        // 5. linear rows and 6. alldifferent groups whose scope changed
        if (n_lin) {
            const uint32_t *mask = I.b + I.h(H_OFF_LIN_MASK);
            if (for_scheduled(I, evs, mask, (int)I.h(H_LIN_MW), [&](int r) {
                    if (lane == 0) evals++;
                    return revise_lin<W>(I, dom, chg, r);
                }))
                return true;
        }
        if (n_ad) {
            const uint32_t *mask = I.b + I.h(H_OFF_AD_MASK);
            if (for_scheduled(I, evs, mask, (int)I.h(H_AD_MW), [&](int g) {
                    if (lane == 0) evals++;
                    return revise_alldiff<W>(I, dom, chg, g);
                }))
                return true;
        }
        __syncwarp();
    }
}

// First-fail: the unfixed variable with the fewest values, lowest index on ties; -1 when
// every variable is fixed.
template <int W>
__device__ __forceinline__ int select_first_fail(const uint32_t *dom, int n) {
    unsigned best = 0xffffffffu;
    for (int v = threadIdx.x & 31; v < n; v += 32) {
        const int pc = dom_popc<W>(dom + v * W);
        if (pc > 1) best = min(best, ((unsigned)pc << 16) | (unsigned)v);
    }
    best = __reduce_min_sync(FULLMASK, best);
    return best == 0xffffffffu ? -1 : (int)(best & 0xffffu);
}

// copy `words` words (a multiple of 4, both pointers 16-byte aligned) with the warp
__device__ __forceinline__ void warp_copy4(uint32_t *dst, const uint32_t *src, int words) {
    const int lane = lane_id();
    uint4 *d = (uint4 *)dst;
    const uint4 *s = (const uint4 *)src;
    for (int i = lane; i < (words >> 2); i += 32) d[i] = s[i];
}
// same, reading through L2 only (records written by other SMs)
__device__ __forceinline__ void warp_copy4_cg(uint32_t *dst, const uint32_t *src, int words) {
    const int lane = lane_id();
    uint4 *d = (uint4 *)dst;
    const uint4 *s = (const uint4 *)src;
    for (int i = lane; i < (words >> 2); i += 32) d[i] = __ldcg(s + i);
}

}  // namespace cubics
