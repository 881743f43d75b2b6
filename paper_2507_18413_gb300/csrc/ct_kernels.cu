// ct_kernels.cu -- CUDA kernels of Compact-Table propagation for sm_103a.
//
// One propagation (Algorithm 1, enforceGAC) is ONE cooperative launch whose
// CTAs step through these phases:
//   plan     Delta_x = lastDom_x & ~dom_x, s_val, s_sup, the delta/reset
//            choice of Algorithm 2 (delta iff |Delta| < |dom|) and the list
//            of supports rows to OR (row codes). For tables whose plan fits in
//            shared memory every CTA computes it for itself; otherwise CTA 0
//            writes it to global memory and a grid barrier follows.
//   update   one warp per 32-chunk segment of currTable (grid-stride):
//            Algorithm 2 on every live 128-bit chunk. The row list is walked
//            flat across variables in batches of 16 (or 8) independent
//            128-bit loads per lane that bypass L1; each variable's OR is complemented on the delta
//            path and AND-ed into the chunk. Changed chunks go to the trail;
//            the segment's live mask (the non-zero index) is rebuilt with one
//            warp ballot.
//   -- grid barrier --
//   probe    Algorithm 1 line 5 (fail when currTable = 0), then one warp per
//            value of s_sup (Algorithm 3 with residues): the residue chunk
//            first; on a miss, two 32-chunk windows after it; values still
//            unresolved go to the hard list.
//   -- grid barrier --
//   scan     one warp per segment holds its live chunks in registers and
//            tests every hard value against them; the last CTA to finish
//            removes the values no chunk supports, stores new residues, writes
//            lastDom and the status block (mapped host memory), and resets the
//            per-call counters for the next call.
// Grid barriers spin with a bounded iteration count; running out sets
// CT_ERR_TIMEOUT and every CTA returns.
#include <cstdint>
#include <cuda_runtime.h>

#include "ct_internal.cuh"

namespace ctk {

namespace {

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

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs resident). The last CTA
// to arrive resets the count and advances the generation; the others poll the
// generation at most kBarrierSpinLimit times. Returns false (after setting
// CT_ERR_TIMEOUT) when the wait ran out.
__device__ bool grid_sync_raw(unsigned* count, unsigned* gen, int* status, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire(gen);
        unsigned arrived;
        // Release this CTA's writes (ordered before by the CTA barrier) and, for
        // the last arrival, acquire everybody else's.
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(count) : "memory");
        if (arrived == gridDim.x - 1) {
            *count = 0u;
            st_release(gen, g + 1u);
        } else {
            unsigned it = 0;
            while (ld_acquire(gen) == g) {
                if (++it > kBarrierSpinLimit) {
                    ok = 0;
                    atomicExch(status, CT_ERR_TIMEOUT);
                    break;
                }
                if (it > 64) __nanosleep(32);
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ bool grid_sync(Ctrl* C, int* s_flag) {
    return grid_sync_raw(&C->bar_count, &C->bar_gen, &C->status, s_flag);
}

struct Smem {
    int32_t codes[kCodeCap];        // row codes of the plan; hard rows in the scan phase
    uint32_t dom[kLocalMaxDW];      // domains at entry, packed in scope order (local plan)
    int32_t k[kLocalMaxArity];      // rows to OR per variable | kCodeDelta
    int32_t rowOff[kLocalMaxArity]; // first code of each variable
    int32_t sup[kLocalMaxArity];    // |dom| > 1
    int32_t scan[kThreads];
    uint32_t cnt[12];
    int flags[8];                   // grow, empty, nval, ndelta, nreset, nsup, nrows
    int flag[4];
    int tr[kWarps];                 // trail entries per warp, then their offsets
    int trBase;
};

enum { kCntLive = 0, kCntLiveIn, kCntWords, kCntTrail, kCntHits, kCntLocal, kCntMiss, kCntPruned, kCntWin };

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

__device__ void plan(const TableDev& T, const VarLayout& V, const uint32_t* __restrict__ dom, int32_t* K,
                     int32_t* rowOff, int32_t* sup, int32_t* codes, uint32_t* domCopy, Smem& sm) {
    const int tid = threadIdx.x;
    if (tid < 8) sm.flags[tid] = 0;
    __syncthreads();
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
        }
        sup[i] = nd > 1;
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

// OR the batch into the running mask; at the last row of a variable apply the
// mask to the accumulator, complemented on the delta path (Algorithm 2).
template <int U>
__device__ __forceinline__ void combine_batch(int q0, int nrows, const int (&code)[U], const uint4 (&v)[U], uint4& m,
                                              uint4& acc) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (q0 + u < nrows) {
            m = or4(m, v[u]);
            if (code[u] & kCodeLast) {
                acc = and4(acc, (code[u] & kCodeDelta) ? not4(m) : m);
                m = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
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

template <int U, bool kGlobal = false>
__device__ __forceinline__ void update_segment(const TableDev& T, int mark, int snapFrom, int snapTo, int seg,
                                               const SegState& S, int nrows, const int32_t* s_codes,
                                               uint32_t* s_cnt, TrailItem& out) {
    const int lane = threadIdx.x & 31;
    const uint32_t mask = S.mask;
    out.need = false;
    // Levels saved since the last call snapshot the index as it is now.
    for (int l = snapFrom + lane; l < snapTo; l += 32) T.levelSeg[(size_t)l * T.nseg + seg] = mask;
    if (mask == 0u) return;
    const bool act = (mask >> lane) & 1u;
    const int w = seg * 32 + lane;
    const uint4 cur = S.cur;
    const int lp = S.lp;
    uint4 acc = make_uint4(~0u, ~0u, ~0u, ~0u), m = make_uint4(0u, 0u, 0u, 0u);
    const uint4* base = T.sup + w;
    const size_t W4 = (size_t)T.W4;
    // Batches of U rows: U independent 128-bit loads in flight per lane; the
    // codes of the next batch are read from shared memory meanwhile.
    int code[U];
#pragma unroll
    for (int u = 0; u < U; ++u) code[u] = u < nrows ? code_at<kGlobal>(T, s_codes, u) : 0;
    for (int q0 = 0; q0 < nrows; q0 += U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_sup_pred(base + (size_t)(code[u] & kCodeRow) * W4, act && q0 + u < nrows);
        int nxt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + U + u;
            nxt[u] = q < nrows ? code_at<kGlobal>(T, s_codes, q) : 0;
        }
        combine_batch<U>(q0, nrows, code, v, m, acc);
#pragma unroll
        for (int u = 0; u < U; ++u) code[u] = nxt[u];
        // Every chunk of this warp is already zero: later masks cannot revive it.
        if (!__any_sync(0xffffffffu, act && nz(and4(acc, cur)))) break;
    }
    const uint4 nv = and4(cur, acc);
    const bool chg = act && !eq4(nv, cur);
    const bool alive = act && nz(nv);
    if (chg) T.curr[w] = nv;
    out.need = chg && mark >= 0 && lp < mark;
    out.w = w;
    out.lp = lp;
    out.cur = cur;
    // The segment's part of the non-zero index: the live chunks after the update.
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

// Trail entries of one round of segments: one reservation per CTA.
__device__ __forceinline__ void trail_round(const TableDev& T, const TrailItem& it, int cap, Smem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nb = __ballot_sync(0xffffffffu, it.need);
    if (lane == 0) sm.tr[warp] = __popc(nb);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < kWarps; ++k) {
            const int c = sm.tr[k];
            sm.tr[k] = tot;
            tot += c;
        }
        int base = 0;
        if (tot) {
            base = atomicAdd(&T.ctrl->trail_top, tot);
            if (base + tot > cap) {
                atomicExch(&T.ctrl->status, CT_ERR_OOM);
                base = -1;
            }
            sm.cnt[kCntTrail] += (uint32_t)tot;
        }
        sm.trBase = base;
    }
    __syncthreads();
    if (it.need && sm.trBase >= 0) {
        const int p = sm.trBase + sm.tr[warp] + __popc(nb & lanemask_lt());
        T.trailKey[p] = make_int2(it.w, it.lp);
        T.trailOld[p] = it.cur;
        T.lastpos[it.w] = p;
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
// A value whose residue missed (whole warp): windows of 32 chunks after the
// residue; a value missed there too goes to the table's hard list.
__device__ __forceinline__ void probe_miss(const TableDev& T, int r, int res, uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31;
    if (T.useResidues) {
        const int W4 = T.W4;
        const uint4* row = T.sup + (size_t)r * W4;
        for (int b = 0; b < kLocalProbes; ++b) {
            if (lane == 0) atomicAdd(&s_cnt[kCntWin], 1u);
            const int c = (int)(((long long)res + 1 + b * 32 + lane) % W4);
            const bool h = nz(and4(ld_sup(row + c), __ldcg(T.curr + c)));
            const unsigned bal = __ballot_sync(0xffffffffu, h);
            if (bal) {
                const int cf = __shfl_sync(0xffffffffu, c, __ffs(bal) - 1);
                if (lane == 0) {
                    T.residue[r] = cf;
                    atomicAdd(&s_cnt[kCntLocal], 1u);
                }
                return;
            }
        }
    }
    if (lane == 0) {
        const unsigned m = atomicAdd(&T.ctrl->nhard, 1u);
        T.hardRow[m] = r;
        T.foundChunk[m] = kNoChunk;
        atomicAdd(&s_cnt[kCntMiss], 1u);
    }
}

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
    probe_miss(T, r, res, s_cnt);
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
                const unsigned bal = __ballot_sync(0xffffffffu, hit[u]);
                if (lane == 0 && bal) atomicMin(&T.foundChunk[m0 + u], seg * 32 + __ffs(bal) - 1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// last CTA: apply Algorithm 3's removals, publish, reset the call counters
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_release_sys(int32_t* p, int32_t v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Run by exactly one CTA once every other CTA is done with the call.
__device__ void finalize(const TableDev& T, const VarLayout& V, uint32_t* __restrict__ dom, Smem& sm, int nh) {
    Ctrl* C = T.ctrl;
    const int tid = threadIdx.x;
    int32_t* H = T.statusBlk;
    if (tid == 0) {
        // Thread 0 may have written control fields just before: make them
        // visible at device scope, then share the status through shared memory.
        __threadfence();
        sm.flag[2] = __ldcg(&C->status);
        sm.cnt[kCntPruned] = 0u;
    }
    __syncthreads();
    const int st = sm.flag[2];
    if (st == CT_OK && nh > 0) {
        uint32_t pruned = 0;
        for (int m = tid; m < nh; m += kThreads) {
            const int r = __ldcg(&T.hardRow[m]);
            const int fc = __ldcg(&T.foundChunk[m]);
            if (fc != kNoChunk) {
                T.residue[r] = fc;
            } else {
                // Algorithm 3 line 4: no live tuple carries the value.
                const int i = T.rowVar[r];
                const int a = r - V.row0(i);
                atomicAnd(&dom[V.off(i) + (a >> 5)], ~(1u << (a & 31)));
                atomicAnd(&T.lastDom[V.ld(i) + (a >> 5)], ~(1u << (a & 31)));
                T.changed[i] = 1;
                ++pruned;
            }
        }
        if (pruned) atomicAdd(&sm.cnt[kCntPruned], pruned);
        __syncthreads();
        if (sm.cnt[kCntPruned]) {
            // Domains of the variables that lost values go to the host.
            uint32_t* outDom = reinterpret_cast<uint32_t*>(H + kStatusHdr + T.nChangedWords);
            for (int q = tid; q < T.nChangedWords; q += kThreads) {
                uint32_t bits = 0u;
                for (int b = 0; b < 32 && q * 32 + b < T.arity; ++b) {
                    const int i = q * 32 + b;
                    if (__ldcg(&T.changed[i])) {
                        bits |= 1u << b;
                        T.changed[i] = 0;
                        for (int k = 0; k < V.nw(i); ++k) outDom[V.ld(i) + k] = __ldcg(&dom[V.off(i) + k]);
                    }
                }
                H[kStatusHdr + q] = (int32_t)bits;
            }
        }
    }
    // Header: one counter per thread, loaded in parallel.
    if (tid < kStatusHdr) {
        int32_t v = 0;
        switch (tid) {
            case kSlotLiveOut: v = (int32_t)__ldcg(&C->live); break;
            case kSlotWordsIn: v = (int32_t)__ldcg(&C->words_in); break;
            case kSlotTrailTop: v = __ldcg(&C->trail_top); break;
            case kSlotMisses: v = __ldcg(&C->misses); break;
            case kSlotPruned: v = (int32_t)sm.cnt[kCntPruned]; break;
            case kSlotHits: v = __ldcg(&C->hits); break;
            case kSlotRowsOred: v = __ldcg(&C->nrows); break;
            case kSlotNval: v = __ldcg(&C->nval); break;
            case kSlotNsup: v = __ldcg(&C->nsup); break;
            case kSlotNdelta: v = __ldcg(&C->ndelta); break;
            case kSlotNreset: v = __ldcg(&C->nreset); break;
            case kSlotTrailAdded: v = __ldcg(&C->trail_added); break;
            case kSlotLiveIn: v = (int32_t)__ldcg(&C->live_in); break;
            case kSlotLocal: v = __ldcg(&C->local_found); break;
            case kSlotHard: v = nh; break;
            case kSlotWindows: v = __ldcg(&C->windows); break;
            case kSlotT1: v = (int32_t)(__ldcg(&C->t[1]) - __ldcg(&C->t[0])); break;
            case kSlotT2: v = (int32_t)(__ldcg(&C->t[2]) - __ldcg(&C->t[0])); break;
            case kSlotT3: v = (int32_t)(__ldcg(&C->t[3]) - __ldcg(&C->t[0])); break;
            case kSlotT4: v = (int32_t)(gtimer() - __ldcg(&C->t[0])); break;
            default: v = 0;
        }
        if (tid != kSlotStatus) H[tid] = v;
    }
    __syncthreads();
    // Reset the per-call counters for the next call (after every read above).
    if (tid == 0) {
        C->live = 0u; C->live_in = 0u; C->words_in = 0u; C->nhard = 0u; C->done = 0u;
        C->hits = 0; C->trail_added = 0; C->local_found = 0; C->misses = 0; C->windows = 0;
        C->nval = 0; C->ndelta = 0; C->nreset = 0; C->nsup = 0; C->nrows = 0;
        C->status = CT_OK;
        // Everything written above reaches the host before the word that publishes it.
        st_release_sys(&H[kSlotStatus], st);
    }
}

// ---------------------------------------------------------------------------
// the propagation kernel
// ---------------------------------------------------------------------------
template <bool kLocal, int U, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
ct_propagate_kernel(const __grid_constant__ TableDev T, uint32_t* __restrict__ dom,
                    const int32_t* __restrict__ domOff, const __grid_constant__ CallParams P) {
    __shared__ Smem sm;
    Ctrl* C = T.ctrl;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    const VarLayout V(T, P.domOff, domOff);
    if (blockIdx.x == 0 && tid == 0) C->t[0] = gtimer();

    // Prologue loads that do not depend on the plan: the warp's first segment
    // and the residue (with its supports chunk) of the first value it probes.
    SegState seg0;
    if (gwarp < T.nseg) seg0 = load_segment(T, gwarp, P.mark);
    int res0 = 0;
    uint4 supRes0 = make_uint4(0u, 0u, 0u, 0u);
    if (T.useResidues && gwarp < T.R && lane == 0) {
        res0 = T.residue[gwarp];
        supRes0 = ld_sup(T.sup + (size_t)gwarp * T.W4 + res0);
    }
    // Levels saved since the last call snapshot lastDom as it is now.
    if (blockIdx.x == 0) {
        for (int l = P.snapFrom; l < P.snapTo; ++l)
            for (int q = tid; q < T.DW; q += kThreads) T.levelDom[(size_t)l * T.DW + q] = T.lastDom[q];
    }

    // plan
    int nrows;
    bool ok;
    if (kLocal) {
        plan(T, V, dom, sm.k, sm.rowOff, sm.sup, sm.codes, sm.dom, sm);
        ok = !(sm.flags[0] || sm.flags[1]);
        nrows = sm.flags[6];
        if (blockIdx.x == 0 && tid == 0) {
            C->nval = sm.flags[2]; C->ndelta = sm.flags[3]; C->nreset = sm.flags[4]; C->nsup = sm.flags[5];
            C->nrows = nrows;
            if (!ok) C->status = sm.flags[0] ? CT_ERR_STATE : CT_INFEASIBLE;
        }
    } else {
        if (blockIdx.x == 0) {
            plan(T, V, dom, T.planK, T.planRowOff, T.varSup, T.codes, nullptr, sm);
            if (tid == 0) {
                C->nval = sm.flags[2]; C->ndelta = sm.flags[3]; C->nreset = sm.flags[4]; C->nsup = sm.flags[5];
                C->nrows = sm.flags[6];
                if (sm.flags[0] || sm.flags[1]) C->status = sm.flags[0] ? CT_ERR_STATE : CT_INFEASIBLE;
            }
        }
        if (!grid_sync(C, &sm.flag[0])) return;
        ok = __ldcg(&C->status) == CT_OK;
        nrows = __ldcg(&C->nrows);
        const int staged = min(nrows, kCodeCap);
        for (int q = tid; q < staged; q += kThreads) sm.codes[q] = __ldcg(&T.codes[q]);
    }
    if (blockIdx.x == 0 && tid == 0) C->t[1] = gtimer();

    if (!ok || nrows == 0) {
        // Nothing to update: currTable stays as it is. Pending level snapshots
        // of the index are still taken.
        for (int seg = gwarp; seg < T.nseg; seg += nwarps) {
            const uint32_t mk = seg == gwarp ? seg0.mask : T.segMask[seg];
            for (int l = P.snapFrom + lane; l < P.snapTo; l += 32) T.levelSeg[(size_t)l * T.nseg + seg] = mk;
        }
        if (!ok) {
            // Domain error or empty domain: publish without filtering.
            if (blockIdx.x == 0) finalize(T, V, dom, sm, 0);
            return;
        }
        if (blockIdx.x == 0 && tid == 0) {
            C->live = (uint32_t)P.prevLive;
            C->live_in = (uint32_t)P.prevLive;
            C->t[2] = C->t[1];
        }
    } else {
        // update (Algorithm 2)
        if (tid < 12) sm.cnt[tid] = 0u;
        __syncthreads();
        const int cap = __ldcg(&C->trail_cap);
        // Rounds of one segment per warp; every warp of a CTA runs every round
        // so that the trail reservation can synchronise the CTA.
        for (int base = blockIdx.x * kWarps; base < T.nseg; base += nwarps) {
            const int seg = base + warp;
            TrailItem it;
            it.need = false;
            if (seg < T.nseg) {
                const SegState S = seg == gwarp ? seg0 : load_segment(T, seg, P.mark);
                update_segment<U>(T, P.mark, P.snapFrom, P.snapTo, seg, S, nrows, sm.codes, sm.cnt, it);
            }
            if (P.mark >= 0) trail_round(T, it, cap, sm);
        }
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&C->live, sm.cnt[kCntLive]);
            atomicAdd(&C->live_in, sm.cnt[kCntLiveIn]);
            atomicAdd(&C->words_in, sm.cnt[kCntWords]);
            if (sm.cnt[kCntTrail]) atomicAdd(&C->trail_added, (int)sm.cnt[kCntTrail]);
        }
        if (!grid_sync(C, &sm.flag[0])) return;
        if (blockIdx.x == 0 && tid == 0) C->t[2] = gtimer();
        // Algorithm 1 line 5: fail when currTable is all zero.
        if (__ldcg(&C->status) != CT_OK || __ldcg(&C->live) == 0u) {
            if (blockIdx.x == 0) {
                if (tid == 0 && __ldcg(&C->status) == CT_OK) C->status = CT_INFEASIBLE;
                __syncthreads();
                finalize(T, V, dom, sm, 0);
            }
            return;
        }
    }

    // residue probes (Algorithm 3)
    if (tid < 12) sm.cnt[tid] = 0u;
    __syncthreads();
    // lastDom := the domains of this call (values pruned below are cleared
    // again by the finalizing CTA).
    if (blockIdx.x == 0) {
        if (kLocal) {
            for (int q = tid; q < T.DW; q += kThreads) T.lastDom[q] = sm.dom[q];
        } else {
            for (int i = tid; i < T.arity; i += kThreads)
                for (int q = 0; q < V.nw(i); ++q) T.lastDom[V.ld(i) + q] = dom[V.off(i) + q];
        }
    }
    for (int r = gwarp; r < T.R; r += nwarps) {
        const int i = __ldg(&T.rowVar[r]);
        const int a = r - V.row0(i);
        bool present;
        if (kLocal) {
            present = sm.sup[i] && ((sm.dom[V.ld(i) + (a >> 5)] >> (a & 31)) & 1u);
        } else {
            present = __ldcg(&T.varSup[i]) && ((dom[V.off(i) + (a >> 5)] >> (a & 31)) & 1u);
        }
        int res = res0;
        uint4 sr = supRes0;
        if (r != gwarp && T.useResidues && present && lane == 0) {
            res = T.residue[r];
            sr = ld_sup(T.sup + (size_t)r * T.W4 + res);
        }
        res = __shfl_sync(0xffffffffu, res, 0);
        probe_row(T, r, present, res, sr, sm.cnt);
    }
    __syncthreads();
    if (tid == 0) {
        if (sm.cnt[kCntHits]) atomicAdd(&C->hits, (int)sm.cnt[kCntHits]);
        if (sm.cnt[kCntLocal]) atomicAdd(&C->local_found, (int)sm.cnt[kCntLocal]);
        if (sm.cnt[kCntMiss]) atomicAdd(&C->misses, (int)sm.cnt[kCntMiss]);
        if (sm.cnt[kCntWin]) atomicAdd(&C->windows, (int)sm.cnt[kCntWin]);
    }
    if (!grid_sync(C, &sm.flag[0])) return;
    if (blockIdx.x == 0 && tid == 0) C->t[3] = gtimer();

    const int nh = (int)__ldcg(&C->nhard);
    if (nh == 0) {
        // Every value kept its support: CTA 0 publishes, the others are done.
        if (blockIdx.x == 0) finalize(T, V, dom, sm, 0);
        return;
    }
    // full scan of the hard values
    {
        const int staged = min(nh, kCodeCap);
        for (int q = tid; q < staged; q += kThreads) sm.codes[q] = __ldcg(&T.hardRow[q]);
        __syncthreads();
        for (int seg = gwarp; seg < T.nseg; seg += nwarps) scan_segment<U>(T, seg, nh, sm.codes);
    }
    // last-block-done
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(&C->done, 1u);
        sm.flag[1] = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!sm.flag[1]) return;
    __threadfence();
    finalize(T, V, dom, sm, nh);
}

// ---------------------------------------------------------------------------
// save / restore of backtrack levels
// ---------------------------------------------------------------------------
__global__ void ct_save_kernel(TableDev T, int level) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    uint32_t* ls = T.levelSeg + (size_t)level * T.nseg;
    uint32_t* ld = T.levelDom + (size_t)level * T.DW;
    for (int s = tid; s < T.nseg; s += nth) ls[s] = T.segMask[s];
    for (int q = tid; q < T.DW; q += nth) ld[q] = T.lastDom[q];
    if (tid == 0) T.ctrl->cur_mark = T.ctrl->trail_top;
}

// Undo the trail entries [mark, top). An entry restores its chunk iff it is the
// first entry of that chunk above the mark (its previous position is below
// the mark), so every chunk is written once and the order does not matter.
__global__ void ct_restore_kernel(TableDev T, int level, int mark, int top, int newMark) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int p = mark + tid; p < top; p += nth) {
        const int2 k = T.trailKey[p];
        if (k.y < mark) {
            T.curr[k.x] = T.trailOld[p];
            T.lastpos[k.x] = k.y;
        }
    }
    const uint32_t* ls = T.levelSeg + (size_t)level * T.nseg;
    const uint32_t* ld = T.levelDom + (size_t)level * T.DW;
    for (int s = tid; s < T.nseg; s += nth) T.segMask[s] = ls[s];
    for (int q = tid; q < T.DW; q += nth) T.lastDom[q] = ld[q];
    if (tid == 0) {
        T.ctrl->trail_top = mark;
        T.ctrl->status = CT_OK;
    }
}

// ---------------------------------------------------------------------------
// A network of tables to its fixpoint in one cooperative launch (Sec. 2:
// propagation removes unsupported values until GAC holds everywhere or a
// failure is found). Rounds are Jacobi steps: every table of the round's work
// list propagates on the same domains (plan, updateTable, failure test,
// filterDomains); their removals are applied together; a table joins the next
// round when another table removed a value of one of its variables. The GAC
// closure is unique, so the order of the propagations does not matter.
// ---------------------------------------------------------------------------

// Entry k of a round's prefix array: the shared-memory copy, or the global
// array itself (read through L2) when the round is too long for the copy.
__device__ __forceinline__ int pre_at(const int32_t* pre, int k, bool global) {
    return global ? __ldcg(pre + k) : pre[k];
}

// Position k of the work list whose prefix range holds u: the largest k < n
// with pre[k] <= u (pre is non-decreasing, pre[0] = 0 <= u). The whole warp
// calls it with the same u. The answer stays in [lo, hi] with pre[lo] <= u;
// each pass samples lo + j * step for j < 32, with 32 * step covering the
// hi - lo + 1 candidates, and keeps the stretch from the last sample <= u to
// the next sample.
__device__ __forceinline__ int find_prefix(const int32_t* pre, int n, int u, bool global) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n - 1;
    while (hi - lo >= 32) {
        const int step = (hi - lo + 32) >> 5;
        const int k = lo + lane * step;
        const unsigned b = __ballot_sync(0xffffffffu, k <= hi && pre_at(pre, k, global) <= u);
        lo += (31 - __clz(b)) * step;
        hi = min(hi, lo + step - 1);
    }
    const int k = lo + lane;
    const unsigned b = __ballot_sync(0xffffffffu, k <= hi && pre_at(pre, k, global) <= u);
    return lo + (31 - __clz(b));
}

// Exclusive prefix of val(work[k]) over k < n into out[0..n] (one CTA).
template <typename F>
__device__ void block_prefix(const int32_t* work, int n, F val, int32_t* out, Smem& sm) {
    const int tid = threadIdx.x;
    const int per = (n + kThreads - 1) / kThreads;
    const int b0 = tid * per, b1 = min(n, b0 + per);
    int sum = 0;
    for (int k = b0; k < b1; ++k) sum += val(__ldcg(&work[k]));
    sm.scan[tid] = sum;
    __syncthreads();
    for (int off = 1; off < kThreads; off <<= 1) {
        const int a = tid >= off ? sm.scan[tid - off] : 0;
        __syncthreads();
        sm.scan[tid] += a;
        __syncthreads();
    }
    int run = sm.scan[tid] - sum;
    for (int k = b0; k < b1; ++k) {
        out[k] = run;
        run += val(__ldcg(&work[k]));
    }
    if (tid == kThreads - 1) out[n] = sm.scan[kThreads - 1];
    __syncthreads();
}

template <int U>
__global__ void __launch_bounds__(kThreads, 2) ct_model_kernel(const __grid_constant__ ModelDev M) {
    __shared__ Smem sm;
    ModelCtrl* C = M.ctrl;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    int32_t* preU = sm.codes;                               // unit prefix of the round (smem copy)
    int32_t* preR = reinterpret_cast<int32_t*>(sm.dom);     // row prefix of the round (smem copy)
    auto sync = [&]() { return grid_sync_raw(&C->bar_count, &C->bar_gen, &C->status, &sm.flag[0]); };
    // optional phase clock: CTA 0 adds the time since its previous mark (a grid
    // barrier ends every phase, so this is the phase's length across the grid)
    uint64_t tmark = (M.phaseNs && blockIdx.x == 0 && tid == 0) ? gtimer() : 0ull;
    auto phase = [&](int p) {
        if (M.phaseNs && blockIdx.x == 0 && tid == 0) {
            const uint64_t now = gtimer();
            M.phaseNs[p] += now - tmark;
            tmark = now;
        }
    };

    if (tid < 12) sm.cnt[tid] = 0u;
    __syncthreads();
    // Trail undos asked for with this launch (one CTA per table): the chunks
    // changed since the level's mark get their value at the mark back, and the
    // index and lastDom their snapshot of the level.
    if (M.nrestores > 0) {
        for (int i = blockIdx.x; i < M.nrestores; i += gridDim.x) {
            const RestoreDesc d = M.restores[i];
            const TableDev& T = M.tabs[d.table];
            for (int p = d.mark + tid; p < d.top; p += kThreads) {
                const int2 k = T.trailKey[p];
                if (k.y < d.mark) {
                    T.curr[k.x] = T.trailOld[p];
                    T.lastpos[k.x] = k.y;
                }
            }
            const uint32_t* ls = T.levelSeg + (size_t)d.level * T.nseg;
            const uint32_t* ld = T.levelDom + (size_t)d.level * T.DW;
            for (int q = tid; q < T.nseg; q += kThreads) T.segMask[q] = ls[q];
            for (int q = tid; q < T.DW; q += kThreads) T.lastDom[q] = ld[q];
            if (tid == 0) {
                T.ctrl->trail_top = d.mark;
                T.ctrl->status = CT_OK;
            }
        }
        if (!sync()) return;
    }
    // Levels saved since each table's last propagation snapshot it as it is now.
    for (int t = blockIdx.x; t < M.ntables; t += gridDim.x) {
        const TableDev& T = M.tabs[t];
        const ModelTabCall cl = M.calls[t];
        for (int l = cl.snapFrom; l < cl.snapTo; ++l) {
            for (int q = tid; q < T.nseg; q += kThreads) T.levelSeg[(size_t)l * T.nseg + q] = __ldcg(&T.segMask[q]);
            for (int q = tid; q < T.DW; q += kThreads) T.levelDom[(size_t)l * T.DW + q] = __ldcg(&T.lastDom[q]);
        }
    }
    int cur = 0, round = 0;
    for (;;) {
        const int nwork = round > 0 ? __ldcg(&C->nnext[round & 1]) : M.nworkIn ? __ldcg(M.nworkIn) : __ldcg(&C->nwork);
        phase(round == 0 ? 0 : 6);
        const int32_t* work = M.work + (size_t)cur * M.ntables;
        int32_t* pruned = M.prunedBy + (size_t)(round & 1) * M.nvars;       // written by this round
        int32_t* prunedNext = M.prunedBy + (size_t)((round + 1) & 1) * M.nvars;
        // the collector of the next round's tables was last read two rounds ago
        if (blockIdx.x == 0 && tid == 0) C->nnext[(round + 1) & 1] = 0;

        // plan (Algorithm 1 lines 1-3), one CTA per table of the round
        for (int k = blockIdx.x; k < nwork; k += gridDim.x) {
            const int t = __ldcg(&work[k]);
            const TableDev& T = M.tabs[t];
            const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
            plan(T, V, M.dom, T.planK, T.planRowOff, T.varSup, T.codes, nullptr, sm);
            if (tid == 0) {
                Ctrl* Tc = T.ctrl;
                Tc->nrows = sm.flags[6];
                Tc->nval = sm.flags[2];
                Tc->ndelta = sm.flags[3];
                Tc->nreset = sm.flags[4];
                Tc->nsup = sm.flags[5];
                if (sm.flags[0]) atomicCAS(&C->status, CT_OK, CT_ERR_STATE);
                else if (sm.flags[1]) M.nodeStatus[t / M.nodeTables] = CT_INFEASIBLE;  // an empty domain
            }
            __syncthreads();
        }
        if (blockIdx.x == 0) {
            block_prefix(work, nwork, [&](int t) { return M.tabs[t].nseg; }, M.unitPrefix, sm);
            block_prefix(work, nwork, [&](int t) { return M.tabs[t].R; }, M.rowPrefix, sm);
        }
        if (!sync()) return;
        phase(1);
        if (__ldcg(&C->status) != CT_OK) break;
        const bool gpre = nwork > kPrefixSmem;
        const int32_t* pU = gpre ? M.unitPrefix : preU;
        const int32_t* pR = gpre ? M.rowPrefix : preR;
        if (!gpre) {
            for (int k = tid; k <= nwork; k += kThreads) {
                preU[k] = __ldcg(&M.unitPrefix[k]);
                preR[k] = __ldcg(&M.rowPrefix[k]);
            }
            __syncthreads();
        }
        const int totalUnits = pre_at(pU, nwork, gpre);
        const int totalRows = pre_at(pR, nwork, gpre);

        // updateTable (Algorithm 2) over (table, segment) units
        for (int u = gwarp; u < totalUnits; u += nwarps) {
            const int k = find_prefix(pU, nwork, u, gpre);
            const int t = __ldcg(&work[k]);
            const TableDev& T = M.tabs[t];
            const int nrows = __ldcg(&T.ctrl->nrows);
            if (nrows == 0) continue;
            const int seg = u - pre_at(pU, k, gpre);
            const int mark = M.calls[t].mark;
            const SegState S = load_segment(T, seg, mark);
            TrailItem it;
            update_segment<U, true>(T, mark, 0, 0, seg, S, nrows, nullptr,
                                    reinterpret_cast<uint32_t*>(&T.ctrl->live), it);
            trail_warp(T, it, __ldcg(&T.ctrl->trail_cap), &C->status);
        }
        if (!sync()) return;
        phase(2);

        if (__ldcg(&C->status) != CT_OK) break;
        // Algorithm 1 line 5: a table whose currTable became zero fails its node;
        // the node's tables leave the work list from the next round on.
        for (int k = blockIdx.x * kThreads + tid; k < nwork; k += gridDim.x * kThreads) {
            const int t = __ldcg(&work[k]);
            const Ctrl* Tc = M.tabs[t].ctrl;
            if (__ldcg(&Tc->nrows) > 0 && __ldcg(&Tc->live) == 0u) M.nodeStatus[t / M.nodeTables] = CT_INFEASIBLE;
        }
        // lastDom := the domains of this round (removals below clear their bits)
        for (int k = blockIdx.x; k < nwork; k += gridDim.x) {
            const int t = __ldcg(&work[k]);
            const TableDev& T = M.tabs[t];
            const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
            for (int i = tid; i < T.arity; i += kThreads)
                for (int q = 0; q < V.nw(i); ++q) T.lastDom[V.ld(i) + q] = __ldcg(&M.dom[V.off(i) + q]);
        }
        // filterDomains (Algorithm 3): the residue test of every (table, row) unit,
        // one unit per lane; a warp then takes its lanes' misses one by one
        // through the windows after the residue, and what misses there too
        // goes to the full scan.
        // rows per warp: up to 32, fewer when that spreads the rows (and their
        // misses) over more warps
        const int rpw = min(32, max(1, (totalRows + nwarps - 1) / nwarps));
        for (int u0 = gwarp * rpw; u0 < totalRows; u0 += nwarps * rpw) {
            const int u = u0 + lane;
            const bool valid = lane < rpw && u < totalRows;
            int k = find_prefix(pR, nwork, u0, gpre);
            while (valid && k + 1 < nwork && pre_at(pR, k + 1, gpre) <= u) ++k;
            bool need = false, hit = false;
            int t = 0, r = 0, res = 0;
            if (valid) {
                t = __ldcg(&work[k]);
                const TableDev& T = M.tabs[t];
                const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
                r = u - pre_at(pR, k, gpre);
                const int i = __ldg(&T.rowVar[r]);
                const int a = r - V.row0(i);
                const bool present =
                    __ldcg(&T.varSup[i]) && ((__ldcg(&M.dom[V.off(i) + (a >> 5)]) >> (a & 31)) & 1u);
                if (present) {
                    if (T.useResidues) {
                        res = T.residue[r];
                        hit = nz(and4(ld_sup(T.sup + (size_t)r * T.W4 + res), __ldcg(T.curr + res)));
                    }
                    need = !hit;
                }
            }
            unsigned miss = __ballot_sync(0xffffffffu, need);
            const int nhit = __popc(__ballot_sync(0xffffffffu, hit));
            if (lane == 0 && nhit) atomicAdd(&sm.cnt[kCntHits], (unsigned)nhit);
            while (miss) {
                const int l = __ffs(miss) - 1;
                miss &= miss - 1u;
                const int tl = __shfl_sync(0xffffffffu, t, l);
                probe_miss(M.tabs[tl], __shfl_sync(0xffffffffu, r, l), __shfl_sync(0xffffffffu, res, l), sm.cnt);
            }
        }
        if (!sync()) return;
        phase(3);

        // full scans of the values whose residues and windows missed
        for (int u = gwarp; u < totalUnits; u += nwarps) {
            const int k = find_prefix(pU, nwork, u, gpre);
            const TableDev& T = M.tabs[__ldcg(&work[k])];
            const int nh = (int)__ldcg(&T.ctrl->nhard);
            if (nh == 0) continue;
            scan_segment<U, true>(T, u - pre_at(pU, k, gpre), nh, nullptr);
        }
        if (!sync()) return;
        phase(4);

        // Algorithm 3 line 4: remove the values no live tuple carries
        for (int k = blockIdx.x; k < nwork; k += gridDim.x) {
            const int t = __ldcg(&work[k]);
            const TableDev& T = M.tabs[t];
            const int nh = (int)__ldcg(&T.ctrl->nhard);
            const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
            for (int m = tid; m < nh; m += kThreads) {
                const int r = __ldcg(&T.hardRow[m]);
                const int fc = __ldcg(&T.foundChunk[m]);
                if (fc != kNoChunk) {
                    T.residue[r] = fc;
                } else {
                    const int i = T.rowVar[r];
                    const int a = r - V.row0(i);
                    atomicAnd(&M.dom[V.off(i) + (a >> 5)], ~(1u << (a & 31)));
                    atomicAnd(&T.lastDom[V.ld(i) + (a >> 5)], ~(1u << (a & 31)));
                    const int v = M.scopeVar[M.scopeBase[t] + i];
                    const int old = atomicCAS(&pruned[v], -1, t);
                    if (old != -1 && old != t) atomicExch(&pruned[v], -2);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (sm.cnt[kCntHits]) atomicAdd(&C->hits, sm.cnt[kCntHits]);
            if (sm.cnt[kCntLocal]) atomicAdd(&C->local, sm.cnt[kCntLocal]);
            if (sm.cnt[kCntMiss]) atomicAdd(&C->hard, sm.cnt[kCntMiss]);
            if (sm.cnt[kCntWin]) atomicAdd(&C->windows, sm.cnt[kCntWin]);
            sm.cnt[kCntHits] = sm.cnt[kCntLocal] = sm.cnt[kCntMiss] = sm.cnt[kCntWin] = 0u;
        }
        if (!sync()) return;
        phase(5);

        // next round (whole grid): every table of a live node that shares a
        // variable another table pruned; the other parity's marks are cleared
        // for the round after
        {
            int32_t* next = M.work + (size_t)(cur ^ 1) * M.ntables;
            int32_t* nnext = &C->nnext[(round + 1) & 1];
            const int gtid = blockIdx.x * kThreads + tid, gth = gridDim.x * kThreads;
            for (int k = gtid; k < nwork; k += gth) {
                Ctrl* Tc = M.tabs[__ldcg(&work[k])].ctrl;
                if (__ldcg(&Tc->nrows) > 0) Tc->live_state = (int32_t)__ldcg(&Tc->live);
                Tc->live = 0u; Tc->live_in = 0u; Tc->words_in = 0u; Tc->nhard = 0u; Tc->nrows = 0;
            }
            for (int t0 = gtid - lane; t0 < M.ntables; t0 += gth) {  // warp-uniform trip count
                const int t = t0 + lane;
                bool dirty = false;
                if (t < M.ntables && __ldcg(&M.nodeStatus[t / M.nodeTables]) == CT_OK) {
                    for (int j = M.scopeBase[t]; j < M.scopeBase[t + 1] && !dirty; ++j) {
                        const int p = __ldcg(&pruned[M.scopeVar[j]]);
                        dirty = p != -1 && p != t;
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, dirty);
                if (bal) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(nnext, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (dirty) next[base + __popc(bal & lanemask_lt())] = t;
                }
            }
            for (int v = gtid; v < M.nvars; v += gth) prunedNext[v] = -1;
            if (blockIdx.x == 0 && tid == 0) {
                C->rounds += 1;
                C->props += nwork;
            }
        }
        cur ^= 1;
        ++round;
        if (!sync()) return;
        if (__ldcg(&C->nnext[round & 1]) == 0) break;
        if (round >= M.maxRounds) {
            if (blockIdx.x == 0 && tid == 0) atomicCAS(&C->status, CT_OK, CT_ERR_TIMEOUT);
            break;
        }
    }

    // publish (CTA 0; every CTA left the loop at the same point)
    if (blockIdx.x != 0) return;
    phase(6);
    __threadfence();
    __syncthreads();
    int32_t* H = M.statusBlk;
    for (int t = tid; t < M.ntables; t += kThreads) {
        Ctrl* Tc = M.tabs[t].ctrl;
        H[kModelHdr + 2 * t] = __ldcg(&Tc->trail_top);
        H[kModelHdr + 2 * t + 1] = __ldcg(&Tc->live_state);
        // leave every table's per-call counters clear
        Tc->live = 0u; Tc->live_in = 0u; Tc->words_in = 0u; Tc->nhard = 0u; Tc->nrows = 0;
        Tc->hits = 0; Tc->local_found = 0; Tc->misses = 0; Tc->windows = 0; Tc->trail_added = 0;
        Tc->status = CT_OK;
    }
    uint32_t* outDom = reinterpret_cast<uint32_t*>(H + kModelHdr + 2 * M.ntables);
    for (int q = tid; q < M.DWg; q += kThreads) outDom[q] = __ldcg(&M.dom[q]);
    const int nnodes = M.ntables / M.nodeTables;
    int32_t* outNode = H + kModelHdr + 2 * M.ntables + M.DWg;
    for (int q = tid; q < nnodes; q += kThreads) {
        outNode[q] = __ldcg(&M.nodeStatus[q]);
        M.nodeStatus[q] = CT_OK;
    }
    for (int v = tid; v < 2 * M.nvars; v += kThreads) M.prunedBy[v] = -1;
    __syncthreads();
    if (tid == 0) {
        const int st = __ldcg(&C->status);
        H[1] = __ldcg(&C->rounds);
        H[2] = __ldcg(&C->props);
        H[3] = (int32_t)__ldcg(&C->hits);
        H[4] = (int32_t)__ldcg(&C->local);
        H[5] = (int32_t)__ldcg(&C->hard);
        H[6] = (int32_t)__ldcg(&C->windows);
        C->hits = C->local = C->hard = C->windows = 0u;
        C->status = CT_OK;
        C->rounds = 0;
        C->props = 0;
        C->nwork = 0;
        phase(7);
        st_release_sys(&H[0], st);
    }
}

// Restores of several tables in one launch: blockIdx.y picks the table.
__global__ void ct_restore_batch_kernel(const TableDev* __restrict__ tabs, const __grid_constant__ RestoreBatch B) {
    const RestoreDesc d = B.d[blockIdx.y];
    const TableDev& T = tabs[d.table];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int p = d.mark + tid; p < d.top; p += nth) {
        const int2 k = T.trailKey[p];
        if (k.y < d.mark) {
            T.curr[k.x] = T.trailOld[p];
            T.lastpos[k.x] = k.y;
        }
    }
    const uint32_t* ls = T.levelSeg + (size_t)d.level * T.nseg;
    const uint32_t* ld = T.levelDom + (size_t)d.level * T.DW;
    for (int s = tid; s < T.nseg; s += nth) T.segMask[s] = ls[s];
    for (int q = tid; q < T.DW; q += nth) T.lastDom[q] = ld[q];
    if (tid == 0) {
        T.ctrl->trail_top = d.mark;
        T.ctrl->status = CT_OK;
    }
}

// Clone j takes the state of source table j % nsrc (blockIdx.y = j - y0).
__global__ void ct_clone_state_kernel(const TableDev* __restrict__ src, const TableDev* __restrict__ dst, int nsrc,
                                      int y0) {
    const int j = y0 + (int)blockIdx.y;
    const TableDev& S = src[j % nsrc];
    const TableDev& D = dst[j];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    const int pad = S.nseg * 32;
    for (int q = tid; q < pad; q += nth) {
        D.curr[q] = S.curr[q];
        D.lastpos[q] = -1;
    }
    for (int q = tid; q < S.nseg; q += nth) D.segMask[q] = S.segMask[q];
    for (int q = tid; q < S.R; q += nth) D.residue[q] = S.residue[q];
    for (int q = tid; q < S.DW; q += nth) D.lastDom[q] = S.lastDom[q];
    for (int q = tid; q < S.arity; q += nth) D.changed[q] = 0;
    if (tid == 0) {
        const int32_t cap = D.ctrl->trail_cap;
        const int32_t live = S.ctrl->live_state;
        int32_t* c = reinterpret_cast<int32_t*>(D.ctrl);
        for (int q = 0; q < (int)(sizeof(Ctrl) / sizeof(int32_t)); ++q) c[q] = 0;
        D.ctrl->cur_mark = -1;
        D.ctrl->trail_cap = cap;
        D.ctrl->live_state = live;
    }
}

struct WordsParam {
    uint32_t w[64];
};

__global__ void ct_set_words_kernel(uint32_t* dst, WordsParam p, int n) {
    const int t = threadIdx.x;
    if (t < n) dst[t] = p.w[t];
}

__global__ void ct_copy_words_kernel(uint32_t* dst, const uint32_t* src, int n) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) dst[q] = src[q];
}

template <bool L, int U, int B>
cudaError_t launch_coop(const TableDev& T, int grid, uint32_t* dom, const int32_t* domOff, const CallParams& P,
                        cudaStream_t s) {
    TableDev t = T;
    CallParams p = P;
    void* args[] = {&t, &dom, (void*)&domOff, &p};
    return cudaLaunchCooperativeKernel((const void*)ct_propagate_kernel<L, U, B>, dim3(grid), dim3(kThreads), args,
                                       0, s);
}

template <bool L, int U, int B>
int coresident() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ct_propagate_kernel<L, U, B>, kThreads, 0) != cudaSuccess)
        return 0;
    return per * sms;
}

}  // namespace

// variant: bit 0 = local plan, bit 1 = wide (8 loads in flight, 3 CTAs per SM)
int max_coresident_blocks(int variant) {
    int r = 0;
    switch (variant & 3) {
        case 0: r = coresident<false, 16, 2>(); break;
        case 1: r = coresident<true, 16, 2>(); break;
        case 2: r = coresident<false, 8, 3>(); break;
        default: r = coresident<true, 8, 3>(); break;
    }
    cudaGetLastError();
    return r;
}

cudaError_t launch_propagate(const TableDev& T, int variant, int grid, uint32_t* dom, const int32_t* domOff,
                             const CallParams& P, cudaStream_t s) {
    switch (variant & 3) {
        case 0: return launch_coop<false, 16, 2>(T, grid, dom, domOff, P, s);
        case 1: return launch_coop<true, 16, 2>(T, grid, dom, domOff, P, s);
        case 2: return launch_coop<false, 8, 3>(T, grid, dom, domOff, P, s);
        default: return launch_coop<true, 8, 3>(T, grid, dom, domOff, P, s);
    }
}

int max_coresident_model_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ct_model_kernel<16>, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per * sms;
}

cudaError_t launch_model(const ModelDev& M, int grid, cudaStream_t s) {
    ModelDev m = M;
    void* args[] = {&m};
    return cudaLaunchCooperativeKernel((const void*)ct_model_kernel<16>, dim3(grid), dim3(kThreads), args, 0, s);
}

cudaError_t launch_restore_batch(const TableDev* tabs, const RestoreBatch& B, cudaStream_t s) {
    if (B.n <= 0) return cudaSuccess;
    ct_restore_batch_kernel<<<dim3(8, B.n), 256, 0, s>>>(tabs, B);
    return cudaGetLastError();
}

cudaError_t launch_clone_state(const TableDev* src, const TableDev* dst, int nsrc, int n, cudaStream_t s) {
    for (int y0 = 0; y0 < n; y0 += 65535) {
        const int ny = (n - y0) < 65535 ? (n - y0) : 65535;
        ct_clone_state_kernel<<<dim3(4, ny), 256, 0, s>>>(src, dst, nsrc, y0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_save(const TableDev& T, int level, cudaStream_t s) {
    const int n = T.nseg > T.DW ? T.nseg : T.DW;
    int grid = (n + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    ct_save_kernel<<<grid, 256, 0, s>>>(T, level);
    return cudaGetLastError();
}

cudaError_t launch_restore(const TableDev& T, int level, int mark, int top, int newMark, cudaStream_t s) {
    int n = top - mark;
    if (T.nseg > n) n = T.nseg;
    if (T.DW > n) n = T.DW;
    int grid = (n + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    ct_restore_kernel<<<grid, 256, 0, s>>>(T, level, mark, top, newMark);
    return cudaGetLastError();
}

cudaError_t launch_set_words(uint32_t* dst, const uint32_t* words, int n, cudaStream_t s) {
    for (int off = 0; off < n; off += 64) {
        WordsParam p;
        const int k = (n - off) < 64 ? (n - off) : 64;
        for (int q = 0; q < k; ++q) p.w[q] = words[off + q];
        ct_set_words_kernel<<<1, 64, 0, s>>>(dst + off, p, k);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_copy_words(uint32_t* dst, const uint32_t* src, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    if (grid > 1024) grid = 1024;
    ct_copy_words_kernel<<<grid, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace ctk
