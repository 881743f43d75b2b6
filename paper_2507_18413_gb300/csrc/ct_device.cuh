// ct_device.cuh -- device building blocks shared by the propagation kernel of
// one table (ct_kernels.cu) and the network fixpoint kernel (ct_model_kernels.cu):
// 128-bit helpers, the bounded grid barrier, the plan of Algorithms 1-2, the
// segment update of Algorithm 2 with its trail, the residue probes of
// Algorithm 3 and the scan of the hard values.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ct_internal.cuh"

namespace ctk {
namespace {

#ifdef CT_PHASE_TRACE
// Diagnostic build only (-DCT_PHASE_TRACE): %globaltimer stamps of thread 0 of
// the first kTraceCtas CTAs at the phase boundaries of the last propagation,
// read with ct_trace_read (one array per translation unit; the propagation
// kernel's is read). The default build has none of this.
constexpr int kTraceCtas = 1024, kTraceStamps = 24;
__device__ unsigned long long g_ct_trace[kTraceCtas * kTraceStamps];
__device__ __forceinline__ unsigned long long gtimer_trace() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define CT_STAMP(k)                                                          \
    do {                                                                     \
        if (threadIdx.x == 0 && blockIdx.x < kTraceCtas)                     \
            g_ct_trace[blockIdx.x * kTraceStamps + (k)] = gtimer_trace();    \
    } while (0)
#else
#define CT_STAMP(k) \
    do {            \
    } while (0)
#endif



__device__ __forceinline__ bool nz(const uint4& v) { return (v.x | v.y | v.z | v.w) != 0u; }

__device__ __forceinline__ uint4 or4(const uint4& a, const uint4& b) {
    return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
}

__device__ __forceinline__ uint4 and4(const uint4& a, const uint4& b) {
    return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ uint4 not4(const uint4& a) { return make_uint4(~a.x, ~a.y, ~a.z, ~a.w); }

__device__ __forceinline__ bool eq4(const uint4& a, const uint4& b) {
    return ((a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w)) == 0u;
}

__device__ __forceinline__ uint32_t nzwords(const uint4& v) {
    return (v.x != 0u) + (v.y != 0u) + (v.z != 0u) + (v.w != 0u);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Read-only 128-bit load of a supports chunk (the supports never change).
__device__ __forceinline__ uint4 ld_sup(const uint4* p) { return __ldg(p); }

// Predicated read-only 128-bit load (zero when `pred` is false), not kept in
// L1 (the supports rows stream through once per call). Written as volatile PTX
// so that a batch of them issues back to back, before any use.
__device__ __forceinline__ uint4 ld_sup_pred(const uint4* p, bool pred) {
    uint4 v;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.b32 q, %5, 0;\n\t"
        "mov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\tmov.b32 %2, 0;\n\tmov.b32 %3, 0;\n\t"
        "@q ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "r"((int)pred));
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Plain (relaxed) read of a word another launch wrote: no ordering imposed on
// the loads that follow.
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs resident). The arrival
// count only grows: barrier k of a launch is complete when the count reaches
// base + k * gridDim.x, where base is the count every launch starts from (the
// last target the previous launch reached, stored by the last arrival of each
// barrier). Thread 0 of every CTA reads base once at the start of the launch
// (no CTA of the launch can store it before this CTA's first arrival, which
// releases that read) and keeps the next target in a register. Waiters poll
// the count itself, so a barrier costs the arrival atomic plus the time for
// the last arrival to reach the count (no second word to publish). Every
// launch must run the same barrier sequence in every CTA. bar_sync returns 0
// (after setting CT_ERR_TIMEOUT) when the wait ran out after `limit` polls, 2
// to the CTA that arrived last (it has acquired every other CTA's writes and
// goes on at once), 1 to the others. The signed difference keeps the test
// valid across the 32-bit wrap.
struct GridBarrier {
    unsigned* count;
    unsigned* base;
    int* status;
    unsigned limit;
    unsigned target;  // count that completes the current barrier (thread 0)
};

__device__ __forceinline__ void bar_init(GridBarrier& b, unsigned* count, unsigned* base, int* status,
                                         unsigned limit) {
    b.count = count;
    b.base = base;
    b.status = status;
    b.limit = limit;
    b.target = threadIdx.x == 0 ? ld_relaxed(base) : 0u;
}

__device__ int bar_sync(GridBarrier& b, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = 1;
        unsigned arrived;
        b.target += gridDim.x;
        // Release this CTA's writes (ordered before by the CTA barrier) and, for
        // the last arrival, acquire everybody else's.
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(b.count) : "memory");
        if (arrived == b.target - 1u) {
            *b.base = b.target;  // read by the next launch only
            r = 2;
        } else {
            unsigned it = 0;
            while ((int)(ld_acquire(b.count) - b.target) < 0) {
                if (++it > b.limit) {
                    r = 0;
                    atomicExch(b.status, CT_ERR_TIMEOUT);
                    break;
                }
                if (it > 64) __nanosleep(32);
            }
        }
        *s_flag = r;
    }
    __syncthreads();
    return *s_flag;
}

struct Smem {
    int32_t codes[kCodeCap];        // row codes of the plan; hard rows in the scan phase
    uint32_t dom[kLocalMaxDW];      // domains at entry, packed in scope order (local plan)
    int32_t k[kLocalMaxArity];      // rows to OR per variable | kCodeDelta
    int32_t rowOff[kLocalMaxArity]; // first code of each variable
    int32_t sup[kLocalMaxArity];    // |dom| > 1
    int32_t nd[kLocalMaxArity];     // |dom| (local plan)
    unsigned long long other[kLocalMaxArity];  // negative tables: product of the other domain sizes (saturated)
    int32_t scan[kThreads];
    uint32_t cnt[12];
    int flags[8];                   // grow, empty, nval, ndelta, nreset, nsup, nrows
    int flag[4];
    int trw[kWarps];  // trail slots of each warp's segment, then their offsets in the CTA's block
    int trBase;       // first trail slot of the CTA's block
};

enum { kCntLive = 0, kCntLiveIn, kCntWords, kCntTrail, kCntHits, kCntLocal, kCntMiss, kCntPruned, kCntWin, kCntTuples };

// ---------------------------------------------------------------------------
// plan: Algorithm 1 lines 1-3 and the row selection of Algorithm 2.
// Writes k/rowOff/sup/codes through generic pointers (shared or global).
// ---------------------------------------------------------------------------
// Layout of scope variable i: from the kernel parameters for small scopes
// (pOff: domain offsets passed as parameters, or null to read domOff).
struct VarLayout {
    const TableDev& T;
    const int32_t* pOff;
    const int32_t* domOff;
    bool small;
    __device__ VarLayout(const TableDev& t, const int32_t* p, const int32_t* d)
        : T(t), pOff(p), domOff(d), small(t.arity <= kParamArity) {}
    __device__ int nw(int i) const { return small ? T.pNW[i] : T.varNW[i]; }
    __device__ int ld(int i) const { return small ? T.pLD[i] : T.varLD[i]; }
    __device__ int row0(int i) const { return small ? T.pRow0[i] : T.varRow0[i]; }
    __device__ int off(int i) const { return (small && pOff) ? pOff[i] : domOff[i]; }
};

// snapFrom/snapTo: levels saved since the last call, whose lastDom snapshot
// (the last-seen domains as they are at entry) this CTA writes from the words
// it loads anyway (an empty range in every CTA but one).
__device__ void plan(const TableDev& T, const VarLayout& V, const uint32_t* __restrict__ dom, int32_t* K,
                     int32_t* rowOff, int32_t* sup, int32_t* codes, uint32_t* domCopy, Smem& sm,
                     int snapFrom = 0, int snapTo = 0) {
    const int tid = threadIdx.x;
    if (tid < 8) sm.flags[tid] = 0;
    __syncthreads();
    CT_STAMP(16);
    for (int i = tid; i < T.arity; i += kThreads) {
        const int nw = V.nw(i);
        const uint32_t* d = dom + V.off(i);
        const uint32_t* l = T.lastDom + V.ld(i);
        int nd = 0, ndel = 0;
        uint32_t grow = 0u;
        for (int q = 0; q < nw; ++q) {
            const uint32_t dv = d[q], lv = l[q];
            grow |= dv & ~lv;
            nd += __popc(dv);
            ndel += __popc(lv & ~dv);
            if (domCopy) domCopy[V.ld(i) + q] = dv;
            for (int lv0 = snapFrom; lv0 < snapTo; ++lv0) T.levelDom[(size_t)lv0 * T.DW + V.ld(i) + q] = lv;
        }
        sup[i] = nd > 1;
        if (i < kLocalMaxArity) sm.nd[i] = nd;
        if (grow) atomicExch(&sm.flags[0], 1);
        if (nd == 0) atomicExch(&sm.flags[1], 1);
        if (nd > 1) atomicAdd(&sm.flags[5], 1);
        int k = 0;
        if (ndel > 0) {
            // Algorithm 2, line 3: the delta mask when |Delta| < |dom| (strict).
            if (ndel < nd) { k = ndel | kCodeDelta; atomicAdd(&sm.flags[3], 1); }
            else { k = nd; atomicAdd(&sm.flags[4], 1); }
            atomicAdd(&sm.flags[2], 1);
        }
        K[i] = k;
    }
    __syncthreads();
    CT_STAMP(17);
    if (sm.flags[0] || sm.flags[1]) {
        if (tid == 0) sm.flags[6] = 0;
        __syncthreads();
        return;
    }
    if (T.arity <= 32) {
        // One warp: lane i owns variable i.
        if (tid < 32) {
            const int k = tid < T.arity ? (K[tid] & kCodeRow) : 0;
            int incl = k;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += a;
            }
            if (tid < T.arity) rowOff[tid] = incl - k;
            if (tid == 31) sm.scan[kThreads - 1] = incl;
        }
        __syncthreads();
    } else {
        // Exclusive scan of the row counts, each thread owning a run of variables.
        const int per = (T.arity + kThreads - 1) / kThreads;
        const int b0 = tid * per, b1 = min(T.arity, b0 + per);
        int sum = 0;
        for (int i = b0; i < b1; ++i) sum += K[i] & kCodeRow;
        sm.scan[tid] = sum;
        __syncthreads();
        for (int off = 1; off < kThreads; off <<= 1) {
            const int a = tid >= off ? sm.scan[tid - off] : 0;
            __syncthreads();
            sm.scan[tid] += a;
            __syncthreads();
        }
        int run = sm.scan[tid] - sum;
        for (int i = b0; i < b1; ++i) {
            rowOff[i] = run;
            run += K[i] & kCodeRow;
        }
        __syncthreads();
    }
    CT_STAMP(18);
    // Codes: the removed values (delta) or the remaining ones (reset).
    for (int i = tid; i < T.arity; i += kThreads) {
        const int k = K[i] & kCodeRow;
        if (k == 0) continue;
        const bool delta = (K[i] & kCodeDelta) != 0;
        const int nw = V.nw(i);
        const uint32_t* d = dom + V.off(i);
        const uint32_t* l = T.lastDom + V.ld(i);
        const int row0 = V.row0(i);
        int out = rowOff[i];
        const int last = out + k - 1;
        for (int q = 0; q < nw; ++q) {
            uint32_t bits = delta ? (l[q] & ~d[q]) : d[q];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                int code = row0 + q * 32 + b;
                if (delta) code |= kCodeDelta;
                if (out == last) code |= kCodeLast;
                codes[out++] = code;
            }
        }
    }
    if (tid == 0) sm.flags[6] = sm.scan[kThreads - 1];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// update: Algorithm 2 on one 32-chunk segment (lane l owns chunk 32*seg + l)
// ---------------------------------------------------------------------------
// Segment state read before the plan is known (it does not depend on it).
struct SegState {
    uint32_t mask;
    uint4 cur;  // dead chunks are zero
    int lp;
};

__device__ __forceinline__ SegState load_segment(const TableDev& T, int seg, int mark) {
    const int w = seg * 32 + (threadIdx.x & 31);
    const bool in = w < T.W4;  // the last segment may be partial
    SegState st;
    st.mask = T.segMask[seg];
    st.cur = in ? T.curr[w] : make_uint4(0u, 0u, 0u, 0u);
    st.lp = (in && mark >= 0) ? T.lastpos[w] : 0x7fffffff;
    return st;
}

struct TrailItem {
    bool need;  // the chunk changed and has no entry above the newest mark yet
    int w;
    int lp;
    uint4 cur;
};

// Row code q: from the shared-memory copy, or from global memory through L2
// when another CTA wrote the plan in this launch (kGlobal).
template <bool kGlobal>
__device__ __forceinline__ int code_at(const TableDev& T, const int32_t* s_codes, int q) {
    if (kGlobal) return __ldcg(&T.codes[q]);
    return q < kCodeCap ? s_codes[q] : __ldcg(&T.codes[q]);
}

// Algorithm 2 on one warp's slice [qa, qb) of a call's row list on one
// segment (lane l holds chunk 32*seg + l). Algorithm 2 ANDs one mask per
// changed variable into currTable, each mask the OR of that variable's rows
// (complemented on the delta path), so the row list may be cut anywhere: a
// slice ANDs the masks of the variables whose rows it holds entirely (the
// return value), and with kSplit leaves in S (warp w) the ORs of the rows of
// a variable cut at its start (head) or at its end (tail), for the warp that
// combines the slices in row order (combine_slices).
//
// Rows go in batches of U independent 128-bit loads per lane, predicated on
// the chunk being live and not kept in L1. Codes in shared memory are read
// at the start of each batch; codes in global memory (kGlobal) are read one
// batch ahead. A slice whose masks already clear every live chunk of the
// segment stops early: the AND of all slices is then zero on every live chunk
// whatever the other slices hold.
template <int U, bool kGlobal, bool kSplit>
__device__ __forceinline__ uint4 slice_rows(const TableDev& T, int seg, bool act, const uint4& cur, int qa, int qb,
                                            const int32_t* s_codes, SliceSmem* S, int w) {
    const int lane = threadIdx.x & 31;
    uint4 acc = make_uint4(~0u, ~0u, ~0u, ~0u);
    int headKind = 0, headDelta = 0, tailKind = 0;
    if (qa < qb) {
        const uint4* base = T.sup + seg * 32 + lane;
        const uint4* baseDelta = T.supDelta + seg * 32 + lane;  // the same rows unless the table has short tuples
        const size_t W4 = (size_t)T.W4;
        bool started = !kSplit || qa == 0 || (code_at<kGlobal>(T, s_codes, qa - 1) & kCodeLast) != 0;
        uint4 m = make_uint4(0u, 0u, 0u, 0u);
        bool cut = false;
        int code[U];
        if (kGlobal) {
#pragma unroll
            for (int u = 0; u < U; ++u) code[u] = qa + u < qb ? code_at<kGlobal>(T, s_codes, qa + u) : 0;
        }
        for (int q0 = qa; q0 < qb; q0 += U) {
            if (!kGlobal) {
#pragma unroll
                for (int u = 0; u < U; ++u) code[u] = q0 + u < qb ? code_at<kGlobal>(T, s_codes, q0 + u) : 0;
            }
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                v[u] = ld_sup_pred(((code[u] & kCodeDelta) ? baseDelta : base) + (size_t)(code[u] & kCodeRow) * W4,
                                   act && q0 + u < qb);
            int nxt[kGlobal ? U : 1];
            if (kGlobal) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + U + u;
                    nxt[kGlobal ? u : 0] = q < qb ? code_at<kGlobal>(T, s_codes, q) : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q0 + u < qb) {
                    m = or4(m, v[u]);
                    if (code[u] & kCodeLast) {
                        const bool dl = (code[u] & kCodeDelta) != 0;
                        if (started) {
                            acc = and4(acc, dl ? not4(m) : m);
                        } else if (kSplit) {
                            S->head[w][lane] = m;
                            headKind = 1;
                            headDelta = dl;
                        }
                        m = make_uint4(0u, 0u, 0u, 0u);
                        started = true;
                    }
                }
            }
            if (kGlobal) {
#pragma unroll
                for (int u = 0; u < U; ++u) code[u] = nxt[kGlobal ? u : 0];
            }
            // Every live chunk of this segment is already zero: later masks cannot revive it.
            if (!__any_sync(0xffffffffu, act && nz(and4(acc, cur)))) {
                cut = true;
                break;
            }
        }
        if (kSplit && !cut) {
            const int lastc = code_at<kGlobal>(T, s_codes, qb - 1);
            if (!(lastc & kCodeLast)) {
                if (started) {
                    S->tail[w][lane] = m;
                    tailKind = 1;
                } else {
                    S->head[w][lane] = m;
                    headKind = 2;
                    headDelta = (lastc & kCodeDelta) != 0;
                }
            }
        }
    }
    if (kSplit) {
        S->acc[w][lane] = acc;
        if (lane == 0) {
            S->headKind[w] = headKind;
            S->headDelta[w] = headDelta;
            S->tailKind[w] = tailKind;
        }
    }
    return acc;
}

// The mask of a segment from the parts of its G slices (warps w0 .. w0+G-1),
// in row order, lane-wise: a head that ends in its slice closes the variable
// the previous slices left open.
__device__ __forceinline__ uint4 combine_slices(const SliceSmem& S, int w0, int G) {
    const int lane = threadIdx.x & 31;
    uint4 acc = make_uint4(~0u, ~0u, ~0u, ~0u), run = make_uint4(0u, 0u, 0u, 0u);
    for (int g = 0; g < G; ++g) {
        const int w = w0 + g;
        acc = and4(acc, S.acc[w][lane]);
        const int hk = S.headKind[w];
        if (hk) {
            run = or4(run, S.head[w][lane]);
            if (hk == 1) {
                acc = and4(acc, S.headDelta[w] ? not4(run) : run);
                run = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (S.tailKind[w]) run = S.tail[w][lane];
    }
    return acc;
}

// The end of Algorithm 2 on one segment, given the AND of its masks: the new
// chunks, the trail item of a changed chunk, and the segment's part of the
// non-zero index rebuilt by one warp ballot. s_cnt: the live/words counters;
// tuples: a negative table's count of valid tuples.
__device__ __forceinline__ void finish_segment(const TableDev& T, int mark, int seg, const SegState& S,
                                               const uint4& acc, uint32_t* s_cnt, uint32_t* tuples,
                                               TrailItem& out) {
    const int lane = threadIdx.x & 31;
    const uint32_t mask = S.mask;
    const bool act = (mask >> lane) & 1u;
    const int w = seg * 32 + lane;
    const uint4 cur = S.cur;
    const uint4 nv = and4(cur, acc);
    const bool chg = act && !eq4(nv, cur);
    const bool alive = act && nz(nv);
    if (chg) T.curr[w] = nv;
    out.need = chg && mark >= 0 && S.lp < mark;
    out.w = w;
    out.lp = S.lp;
    out.cur = cur;
    if (T.negative) {
        // negative tables filter by counts: the valid tuples left
        uint32_t tc = act ? __popc(nv.x) + __popc(nv.y) + __popc(nv.z) + __popc(nv.w) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tc += __shfl_xor_sync(0xffffffffu, tc, o);
        if (lane == 0 && tc) atomicAdd(tuples, tc);
    }
    const uint32_t nmask = __ballot_sync(0xffffffffu, alive);
    uint32_t words = nzwords(cur);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) words += __shfl_xor_sync(0xffffffffu, words, o);
    if (lane == 0) {
        if (nmask != mask) T.segMask[seg] = nmask;
        atomicAdd(&s_cnt[kCntLive], (uint32_t)__popc(nmask));
        atomicAdd(&s_cnt[kCntLiveIn], (uint32_t)__popc(mask));
        atomicAdd(&s_cnt[kCntWords], words);
    }
}

// Algorithm 2 on one segment by one warp (the whole row list): the network kernel's update.
template <int U, bool kGlobal = false>
__device__ __forceinline__ void update_segment(const TableDev& T, int mark, int snapFrom, int snapTo, int seg,
                                               const SegState& S, int nrows, const int32_t* s_codes,
                                               uint32_t* s_cnt, uint32_t* tuples, TrailItem& out) {
    const int lane = threadIdx.x & 31;
    out.need = false;
    // Levels saved since the last call snapshot the index as it is now.
    for (int l = snapFrom + lane; l < snapTo; l += 32) T.levelSeg[(size_t)l * T.nseg + seg] = S.mask;
    if (S.mask == 0u) return;
    const uint4 acc = slice_rows<U, kGlobal, false>(T, seg, (S.mask >> lane) & 1u, S.cur, 0, nrows, s_codes, nullptr, 0);
    finish_segment(T, mark, seg, S, acc, s_cnt, tuples, out);
}

// Trail slots of a round of segments. Each segment's warp counts one slot for
// every live chunk whose newest entry lies below the newest mark (the chunks
// that need an entry if they change); one atomic per CTA reserves the block
// before the rows are read, so its latency hides behind the row loads.
// trail_write fills the slots of the chunks that changed and gives the others
// an unused key (previous position INT_MAX, which no undo takes for a chunk
// below its mark).
struct TrailSlots {
    uint32_t cand;  // lanes holding a slot
    int base;       // the warp's first slot
};

__device__ __forceinline__ void trail_write(const TableDev& T, const TrailSlots& R, const TrailItem& it, int cap,
                                            uint32_t* s_cnt) {
    if (!R.cand) return;
    const int lane = threadIdx.x & 31;
    const int base = __shfl_sync(0xffffffffu, R.base, 0);
    const int n = __popc(R.cand);
    if (base + n > cap) {
        if (lane == 0) atomicExch(&T.ctrl->status, CT_ERR_OOM);
        return;
    }
    if (lane == 0) atomicAdd(&s_cnt[kCntTrail], (uint32_t)n);
    if ((R.cand >> lane) & 1u) {
        const int p = base + __popc(R.cand & lanemask_lt());
        if (it.need) {
            T.trailKey[p] = make_int2(it.w, it.lp);
            T.trailOld[p] = it.cur;
            T.lastpos[it.w] = p;
        } else {
            T.trailKey[p] = make_int2(-1, 0x7fffffff);
        }
    }
}

// Trail entries of one warp: one reservation per warp (used when the CTA's
// warps work on different tables).
__device__ __forceinline__ void trail_warp(const TableDev& T, const TrailItem& it, int cap, int* status) {
    const int lane = threadIdx.x & 31;
    const uint32_t nb = __ballot_sync(0xffffffffu, it.need);
    if (!nb) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&T.ctrl->trail_top, __popc(nb));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + __popc(nb) > cap) {
        if (lane == 0) atomicCAS(status, CT_OK, CT_ERR_OOM);
        return;
    }
    if (it.need) {
        const int p = base + __popc(nb & lanemask_lt());
        T.trailKey[p] = make_int2(it.w, it.lp);
        T.trailOld[p] = it.cur;
        T.lastpos[it.w] = p;
    }
}

// ---------------------------------------------------------------------------
// probe: Algorithm 3 with residues, a warp per value whose residue missed
// ---------------------------------------------------------------------------
// Chunk c of currTable as this call's update leaves it (Algorithm 2), for a
// filter that runs beside the update: the chunk as loaded AND-ed with the
// call's mask at c, the AND over the changed variables of the OR of their rows
// (complemented on the delta path), rows as the update reads them. The load
// may see the chunk before or after the warp that owns it stores the update:
// the update stores new = old & M, and new & M = new, word by word, so a load
// that sees part of the store gives the new chunk too. E >= the call's rows.
template <int E>
__device__ __forceinline__ uint4 chunk_after(const TableDev& T, const int32_t* codes, int nrows, int c) {
    const uint4 cur = __ldcg(T.curr + c);
    uint4 v[E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
        const int code = u < nrows ? codes[u] : 0;
        v[u] = ld_sup_pred(((code & kCodeDelta) ? T.supDelta : T.sup) + (size_t)(code & kCodeRow) * T.W4 + c,
                           u < nrows);
    }
    uint4 acc = make_uint4(~0u, ~0u, ~0u, ~0u), m = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < E; ++u) {
        if (u < nrows) {
            const int code = codes[u];  // (shared memory: read again rather than held)
            m = or4(m, v[u]);
            if (code & kCodeLast) {
                acc = and4(acc, (code & kCodeDelta) ? not4(m) : m);
                m = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
    return and4(cur, acc);
}

// currTable chunk c for a probe: as stored (kE = 0, after the update's
// barrier), or recomputed from the call's rows beside the update (kE rows).
template <int kE>
__device__ __forceinline__ uint4 probe_chunk(const TableDev& T, const int32_t* codes, int nrows, int c) {
    if constexpr (kE > 0) return chunk_after<kE>(T, codes, nrows, c);
    else return __ldcg(T.curr + c);
}

// Position of the k-th (0-based) set bit of m (k < popcount(m)): halve the
// word, keeping the half that holds it.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Outcomes of the window search of a residue miss.
enum { kProbeFound = 1, kProbeGone = 0, kProbeUndecided = -1 };

// A value whose residue missed (whole warp, r and res uniform): Algorithm 3's
// search for a support over the live chunks (the non-zero index) that follow
// the residue in cyclic order (kLive), 32 chunks per window, at most
// kProbes windows over at most kWindowGroups x 32 index segments; without
// kLive, the chunks that follow the residue, dead or alive. Found: the residue
// moves there (kProbeFound). Not found with every live chunk tested: the value
// has no support (kProbeGone). Else kProbeUndecided: a full scan decides.
// (Measured against windows of the chunks that follow the residue, dead or
// alive: the same on the dense bench stream, 8-10% more search nodes per
// second in the batched search.)
template <bool kLive, int kProbes = kLocalProbes, int kE = 0>
__device__ __forceinline__ int probe_windows(const TableDev& T, int r, int res, uint32_t* s_cnt,
                                             const int32_t* codes = nullptr, int nrows = 0) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    bool complete = false;
    if (!kLive && T.useResidues) {
        // the chunks that follow the residue, dead or alive: two windows per
        // round of loads, tested in order
        const int W4 = T.W4;
        const uint4* row = T.sup + (size_t)r * W4;
        // (one window per round when the chunks are recomputed from more than
        // four rows: their row loads)
        constexpr int kStep = kE > 4 ? 1 : 2;
        for (int b = 0; b < kProbes; b += kStep) {
            const int c0 = (int)(((long long)res + 1 + b * 32 + lane) % W4);
            const int c1 = (int)(((long long)res + 1 + (b + 1) * 32 + lane) % W4);
            const bool two = kStep == 2 && b + 1 < kProbes;
            const uint4 s0 = ld_sup(row + c0), t0 = probe_chunk<kE>(T, codes, nrows, c0);
            uint4 s1 = make_uint4(0u, 0u, 0u, 0u), t1 = s1;
            if (two) {
                s1 = ld_sup(row + c1);
                t1 = probe_chunk<kE>(T, codes, nrows, c1);
            }
            for (int k = 0; k < (two ? 2 : 1); ++k) {
                if (lane == 0) atomicAdd(&s_cnt[kCntWin], 1u);
                const int c = k ? c1 : c0;
                const unsigned bal = __ballot_sync(FULL, k ? nz(and4(s1, t1)) : nz(and4(s0, t0)));
                if (bal) {
                    const int cf = __shfl_sync(FULL, c, __ffs(bal) - 1);
                    if (lane == 0) {
                        T.residue[r] = cf;
                        atomicAdd(&s_cnt[kCntLocal], 1u);
                    }
                    return kProbeFound;
                }
            }
        }
    } else if (T.useResidues) {
        const uint4* row = T.sup + (size_t)r * T.W4;
        const int nseg = T.nseg;
        const int s0 = res >> 5, b0 = res & 31;
        const uint32_t above = b0 == 31 ? 0u : (0xffffffffu << (b0 + 1));
        const uint32_t below = (1u << b0) - 1u;
        // virtual segments: s0 (chunks above res), s0+1, ..., s0-1 (cyclic), s0 (chunks below res)
        const int nvirt = nseg + 1;
        int tested = 0;
        complete = true;
        for (int g = 0, v0 = 0; v0 < nvirt && complete; ++g, v0 += 32) {
            if (g == kWindowGroups || tested >= 32 * kProbes) {
                complete = false;
                break;
            }
            const int v = v0 + lane;
            uint32_t mk = 0u;
            int sg = 0;
            if (v < nvirt) {
                sg = s0 + v;
                if (sg >= nseg) sg -= nseg;
                mk = __ldcg(&T.segMask[sg]);
                if (v == 0) mk &= above;
                else if (v == nseg) mk &= below;
            }
            const int c = __popc(mk);
            int inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += t;
            }
            const int total = __shfl_sync(FULL, inc, 31);
            for (int q0 = 0; q0 < total; q0 += 32) {
                if (tested >= 32 * kProbes) {
                    complete = false;
                    break;
                }
                if (lane == 0) atomicAdd(&s_cnt[kCntWin], 1u);
                const int q = q0 + lane;
                // the lane whose segment holds live chunk q of the group: smallest j with inc_j > q
                int lo = 0, hi = 31;
#pragma unroll
                for (int it = 0; it < 5; ++it) {
                    const int mid = (lo + hi) >> 1;
                    if (__shfl_sync(FULL, inc, mid) > q) hi = mid;
                    else lo = mid + 1;
                }
                const uint32_t mj = __shfl_sync(FULL, mk, lo);
                const int before = __shfl_sync(FULL, inc, lo) - __shfl_sync(FULL, c, lo);
                const int sj = __shfl_sync(FULL, sg, lo);
                bool h = false;
                int chunk = 0;
                if (q < total) {
                    chunk = sj * 32 + nth_set_bit(mj, q - before);
                    h = nz(and4(ld_sup(row + chunk), probe_chunk<kE>(T, codes, nrows, chunk)));
                }
                tested += min(32, total - q0);
                const unsigned bal = __ballot_sync(FULL, h);
                if (bal) {
                    const int cf = __shfl_sync(FULL, chunk, __ffs(bal) - 1);
                    if (lane == 0) {
                        T.residue[r] = cf;
                        atomicAdd(&s_cnt[kCntLocal], 1u);
                    }
                    return kProbeFound;
                }
            }
        }
    }
    return complete ? kProbeGone : kProbeUndecided;
}

// A residue miss searched by probe_windows; a value not found goes to the
// hard list, marked kNoSupport when it has no support (removed without a
// scan; a scan keeps the mark, atomicMin), else for the full scan.
__device__ __forceinline__ void note_probe(const TableDev& T, int r, int o, uint32_t* s_cnt) {
    if (o != kProbeFound && (threadIdx.x & 31) == 0) {
        const bool complete = o == kProbeGone;
        const unsigned m = atomicAdd(&T.ctrl->nhard, 1u);
        T.hardRow[m] = r;
        T.foundChunk[m] = complete ? kNoSupport : kNoChunk;
        if (!complete) {
            atomicAdd(&T.ctrl->nscan, 1);
            atomicAdd(&s_cnt[kCntMiss], 1u);
        }
    }
}

template <bool kLive, int kProbes = kLocalProbes, int kE = 0>
__device__ __forceinline__ void probe_miss(const TableDev& T, int r, int res, uint32_t* s_cnt,
                                           const int32_t* codes = nullptr, int nrows = 0) {
    note_probe(T, r, probe_windows<kLive, kProbes, kE>(T, r, res, s_cnt, codes, nrows), s_cnt);
}

// Whole warp: wait (bounded) until every CTA of the launch has released its
// part of the update (Ctrl::upd_done); false when the wait ran out, with
// CT_ERR_TIMEOUT set in the control block.
__device__ __forceinline__ bool wait_update_done(Ctrl* C, unsigned limit) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        unsigned it = 0;
        while (ld_acquire(&C->upd_done) < gridDim.x) {
            if (++it > limit) {
                ok = false;
                atomicExch(&C->status, CT_ERR_TIMEOUT);
                break;
            }
            if (it > 64) __nanosleep(32);
        }
    }
    // lane 0's acquire, then a warp barrier (which orders memory among the
    // lanes): every lane's later loads see the released update
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <bool kLive>
__device__ __forceinline__ void probe_row(const TableDev& T, int r, bool present, int res, uint4 supRes,
                                          uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31;
    if (!present) return;
    if (T.useResidues) {
        bool hit = false;
        if (lane == 0) hit = nz(and4(supRes, __ldcg(T.curr + res)));
        if (__shfl_sync(0xffffffffu, hit, 0)) {
            if (lane == 0) atomicAdd(&s_cnt[kCntHits], 1u);
            return;
        }
    }
    probe_miss<kLive>(T, r, res, s_cnt);
}

// ---------------------------------------------------------------------------
// scan: the hard values against the live chunks of one segment
// ---------------------------------------------------------------------------
template <int U, bool kGlobal = false>
__device__ __forceinline__ void scan_segment(const TableDev& T, int seg, int nh, const int32_t* s_rows) {
    const int lane = threadIdx.x & 31;
    const uint32_t mask = __ldcg(&T.segMask[seg]);
    if (mask == 0u) return;
    const bool act = (mask >> lane) & 1u;
    const int w = seg * 32 + lane;
    const uint4 cur = act ? __ldcg(T.curr + w) : make_uint4(0u, 0u, 0u, 0u);
    const size_t W4 = (size_t)T.W4;
    for (int m0 = 0; m0 < nh; m0 += U) {
        bool hit[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int mm = m0 + u;
            hit[u] = false;
            if (act && mm < nh) {
                const int r = (!kGlobal && mm < kCodeCap) ? s_rows[mm] : __ldcg(&T.hardRow[mm]);
                hit[u] = nz(and4(ld_sup(T.sup + (size_t)r * W4 + w), cur));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (m0 + u < nh) {
                // any supporting chunk is a valid new residue: whichever
                // segment's store lands last stays (a plain store: no
                // round trip and no contended atomic per value)
                const unsigned bal = __ballot_sync(0xffffffffu, hit[u]);
                if (lane == 0 && bal) T.foundChunk[m0 + u] = seg * 32 + __ffs(bal) - 1;
            }
        }
    }
}

// Negative tables: the valid tuples carrying each hard value, summed over the
// live chunks of one segment (foundChunk[m] holds the count).
__device__ __forceinline__ void count_segment(const TableDev& T, int seg, int nh, const int32_t* s_rows) {
    const int lane = threadIdx.x & 31;
    const uint32_t mask = __ldcg(&T.segMask[seg]);
    if (mask == 0u) return;
    const bool act = (mask >> lane) & 1u;
    const int w = seg * 32 + lane;
    const uint4 cur = act ? __ldcg(T.curr + w) : make_uint4(0u, 0u, 0u, 0u);
    const size_t W4 = (size_t)T.W4;
    for (int m = 0; m < nh; ++m) {
        const int r = m < kCodeCap && s_rows ? s_rows[m] : __ldcg(&T.hardRow[m]);
        uint32_t c = 0u;
        if (act) {
            const uint4 v = and4(ld_sup(T.sup + (size_t)r * W4 + w), cur);
            c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) atomicAdd(&T.foundChunk[m], (int)c);
    }
}

__device__ __forceinline__ void st_release_sys(int32_t* p, int32_t v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace
}  // namespace ctk
