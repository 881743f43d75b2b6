// ct_kernels.cu -- CUDA kernels of Compact-Table propagation for sm_103a.
//
// One propagation (Algorithm 1, enforceGAC) is three launches on the table's
// stream:
//   plan    1 CTA.  Change detection: Delta_x = lastDom_x & ~dom_x, s_val,
//                   s_sup, the delta/reset choice of Algorithm 2 (delta iff
//                   |Delta| < |dom|) and the list of supports rows to OR.
//   update  one warp per index segment. Algorithm 2 for every live chunk:
//                   the OR of the planned rows per changed variable
//                   (complemented on the delta path), AND-ed together and
//                   into currTable; changed chunks go to the trail; the
//                   segment's index is compacted with warp ballots (survivors
//                   first, removed chunks after them, so that a restore only
//                   resets the count). The last CTA to finish tests
//                   currTable = 0 (failure) and probes the residue of every
//                   value of s_sup (Algorithm 3, residues of CT).
//   scan    one warp per index segment. Values whose residue missed are
//                   searched in the live chunks (128-bit loads, the segment's
//                   currTable chunks held in registers); the last CTA removes
//                   the values nobody supports, stores new residues, writes
//                   lastDom and the status block.
// There is no spin-wait anywhere: cross-CTA completion uses the
// last-block-done pattern (fence + atomic ticket).
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

// Read-only, keep-in-L1 128-bit load of a supports chunk.
__device__ __forceinline__ uint4 ld_sup(const uint4* p) { return __ldg(p); }

__device__ void write_header(const TableDev& T, int status) {
    Ctrl* C = T.ctrl;
    int32_t* h = T.statusBlk;
    h[kSlotStatus] = status;
    h[kSlotLiveOut] = (int32_t)__ldcg(&C->live);
    h[kSlotWordsIn] = (int32_t)__ldcg(&C->words_in);
    h[kSlotTrailTop] = __ldcg(&C->trail_top);
    h[kSlotMisses] = (int32_t)__ldcg(&C->nmiss);
    h[kSlotPruned] = __ldcg(&C->pruned);
    h[kSlotHits] = __ldcg(&C->hits);
    h[kSlotRowsOred] = __ldcg(&C->nrows);
    h[kSlotNval] = __ldcg(&C->nval);
    h[kSlotNsup] = __ldcg(&C->nsup);
    h[kSlotNdelta] = __ldcg(&C->ndelta);
    h[kSlotNreset] = __ldcg(&C->nreset);
    h[kSlotTrailAdded] = __ldcg(&C->trail_added);
    h[kSlotLiveIn] = (int32_t)__ldcg(&C->live_in);
}

// ---------------------------------------------------------------------------
// plan: Algorithm 1 lines 1-3 plus the row selection of Algorithm 2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPlanThreads)
ct_plan_kernel(TableDev T, const uint32_t* __restrict__ dom, const int32_t* __restrict__ domOff) {
    __shared__ int32_t s_k[kMaxArity];     // rows to OR for each variable (0 if unchanged)
    __shared__ int32_t s_mode[kMaxArity];
    __shared__ int32_t s_rowOff[kMaxArity];
    __shared__ int32_t s_grpOff[kMaxArity];
    __shared__ int32_t s_scanA[kPlanThreads], s_scanB[kPlanThreads];
    __shared__ int s_grow, s_empty, s_nval, s_ndelta, s_nreset, s_nsup;

    Ctrl* C = T.ctrl;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_grow = 0; s_empty = 0; s_nval = 0; s_ndelta = 0; s_nreset = 0; s_nsup = 0;
        C->status = CT_OK;
        C->live = 0u; C->live_in = 0u; C->words_in = 0u; C->nmiss = 0u;
        C->done_update = 0u; C->done_scan = 0u;
        C->hits = 0; C->pruned = 0; C->trail_added = 0;
    }
    __syncthreads();

    for (int i = tid; i < T.arity; i += kPlanThreads) {
        const int nw = T.varNW[i];
        const uint32_t* d = dom + domOff[i];
        const uint32_t* l = T.lastDom + T.varLD[i];
        int nd = 0, ndel = 0;
        uint32_t grow = 0u;
        for (int q = 0; q < nw; ++q) {
            const uint32_t dv = d[q], lv = l[q];
            grow |= dv & ~lv;
            nd += __popc(dv);
            ndel += __popc(lv & ~dv);
        }
        T.changed[i] = 0;
        T.varSup[i] = nd > 1;
        if (grow) atomicExch(&s_grow, 1);
        if (nd == 0) atomicExch(&s_empty, 1);
        if (nd > 1) atomicAdd(&s_nsup, 1);
        int k = 0, mode = kModeReset;
        if (ndel > 0) {
            // Algorithm 2, line 3: the delta mask when |Delta| < |dom| (strict).
            if (ndel < nd) { k = ndel; mode = kModeDelta; atomicAdd(&s_ndelta, 1); }
            else { k = nd; mode = kModeReset; atomicAdd(&s_nreset, 1); }
            atomicAdd(&s_nval, 1);
        }
        s_k[i] = k;
        s_mode[i] = mode;
    }
    __syncthreads();
    // A grown domain (including stray bits above dom_size) or an empty one ends
    // the call here, before any row is listed.
    if (s_grow || s_empty) {
        if (tid == 0) {
            C->nval = s_nval; C->ndelta = s_ndelta; C->nreset = s_nreset; C->nsup = s_nsup;
            C->ngroups = 0; C->nrows = 0;
            C->status = s_grow ? CT_ERR_STATE : CT_INFEASIBLE;
        }
        return;
    }

    // Exclusive scans of k (row offsets) and of [k > 0] (group slots), each
    // thread owning a contiguous run of variables.
    const int per = (T.arity + kPlanThreads - 1) / kPlanThreads;
    const int b0 = tid * per, b1 = min(T.arity, b0 + per);
    int sumA = 0, sumB = 0;
    for (int i = b0; i < b1; ++i) { sumA += s_k[i]; sumB += s_k[i] > 0; }
    s_scanA[tid] = sumA;
    s_scanB[tid] = sumB;
    __syncthreads();
    for (int off = 1; off < kPlanThreads; off <<= 1) {
        int a = 0, b = 0;
        if (tid >= off) { a = s_scanA[tid - off]; b = s_scanB[tid - off]; }
        __syncthreads();
        s_scanA[tid] += a;
        s_scanB[tid] += b;
        __syncthreads();
    }
    int runA = s_scanA[tid] - sumA, runB = s_scanB[tid] - sumB;
    for (int i = b0; i < b1; ++i) {
        s_rowOff[i] = runA;
        s_grpOff[i] = runB;
        runA += s_k[i];
        runB += s_k[i] > 0;
    }
    __syncthreads();

    // Rows of each changed variable: the removed values (delta) or the
    // remaining ones (reset).
    for (int i = tid; i < T.arity; i += kPlanThreads) {
        const int k = s_k[i];
        if (k == 0) continue;
        const int nw = T.varNW[i];
        const uint32_t* d = dom + domOff[i];
        const uint32_t* l = T.lastDom + T.varLD[i];
        const int row0 = T.varRow0[i];
        int out = s_rowOff[i];
        for (int q = 0; q < nw; ++q) {
            uint32_t bits = (s_mode[i] == kModeDelta) ? (l[q] & ~d[q]) : d[q];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                T.planRows[out++] = row0 + q * 32 + b;
            }
        }
        Group g;
        g.row_begin = s_rowOff[i];
        g.row_count = k;
        g.mode = s_mode[i];
        g.var = i;
        T.groups[s_grpOff[i]] = g;
    }
    if (tid == kPlanThreads - 1) {
        C->ngroups = s_scanB[kPlanThreads - 1];
        C->nrows = s_scanA[kPlanThreads - 1];
    }
    __syncthreads();
    if (tid == 0) { C->nval = s_nval; C->ndelta = s_ndelta; C->nreset = s_nreset; C->nsup = s_nsup; }
}

// ---------------------------------------------------------------------------
// update: Algorithm 2 over the live chunks, trail, index compaction; the last
// CTA tests for failure and probes residues.
// ---------------------------------------------------------------------------
template <int E>
__global__ void __launch_bounds__(512)
ct_update_kernel(TableDev T, const uint32_t* __restrict__ dom, const int32_t* __restrict__ domOff) {
    Ctrl* C = T.ctrl;
    if (C->status != CT_OK) return;

    __shared__ uint32_t s_live, s_livein, s_words, s_trail;
    __shared__ int s_last;
    if (threadIdx.x == 0) { s_live = 0u; s_livein = 0u; s_words = 0u; s_trail = 0u; }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int seg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ngroups = C->ngroups;

    if (seg < T.nseg) {
        const int c = T.segCnt[seg];
        const int base = seg * T.S;
        int32_t* idx = T.idx + base;
        if (ngroups == 0) {
            if (lane == 0) { atomicAdd(&s_live, (uint32_t)c); atomicAdd(&s_livein, (uint32_t)c); }
        } else {
            bool act[E];
            int w[E];
            uint4 cur[E], acc[E];
            uint32_t words = 0u;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                act[e] = e * 32 + lane < c;
                w[e] = act[e] ? idx[e * 32 + lane] : 0;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                cur[e] = act[e] ? T.curr[w[e]] : make_uint4(0u, 0u, 0u, 0u);
                acc[e] = make_uint4(~0u, ~0u, ~0u, ~0u);
                words += nzwords(cur[e]);
            }
            const size_t W4 = (size_t)T.W4;
            for (int g = 0; g < ngroups; ++g) {
                const Group G = T.groups[g];
                const int32_t* rows = T.planRows + G.row_begin;
                uint4 m[E];
#pragma unroll
                for (int e = 0; e < E; ++e) m[e] = make_uint4(0u, 0u, 0u, 0u);
                int q = 0;
                for (; q + 4 <= G.row_count; q += 4) {
                    const uint4* r0 = T.sup + (size_t)rows[q] * W4;
                    const uint4* r1 = T.sup + (size_t)rows[q + 1] * W4;
                    const uint4* r2 = T.sup + (size_t)rows[q + 2] * W4;
                    const uint4* r3 = T.sup + (size_t)rows[q + 3] * W4;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (act[e]) {
                            const uint4 a0 = ld_sup(r0 + w[e]);
                            const uint4 a1 = ld_sup(r1 + w[e]);
                            const uint4 a2 = ld_sup(r2 + w[e]);
                            const uint4 a3 = ld_sup(r3 + w[e]);
                            m[e] = or4(m[e], or4(or4(a0, a1), or4(a2, a3)));
                        }
                    }
                }
                for (; q < G.row_count; ++q) {
                    const uint4* r0 = T.sup + (size_t)rows[q] * W4;
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (act[e]) m[e] = or4(m[e], ld_sup(r0 + w[e]));
                }
                const bool delta = G.mode == kModeDelta;
                bool any = false;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    acc[e] = and4(acc[e], delta ? not4(m[e]) : m[e]);
                    any |= act[e] && nz(and4(acc[e], cur[e]));
                }
                // Every chunk of this warp is already zero: later masks cannot revive it.
                if (!__any_sync(0xffffffffu, any)) break;
            }

            const int mark = C->cur_mark;
            bool alive[E], need[E];
            int prev[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint4 nv = and4(cur[e], acc[e]);
                const bool chg = act[e] && !eq4(nv, cur[e]);
                alive[e] = act[e] && nz(nv);
                if (chg) T.curr[w[e]] = nv;
                prev[e] = (chg && mark >= 0) ? T.lastpos[w[e]] : 0x7fffffff;
                need[e] = chg && mark >= 0 && prev[e] < mark;
            }

            // Trail: one reservation per warp.
            uint32_t nb[E];
            int ntr = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) { nb[e] = __ballot_sync(0xffffffffu, need[e]); ntr += __popc(nb[e]); }
            if (ntr) {
                int tb = 0;
                if (lane == 0) tb = atomicAdd(&C->trail_top, ntr);
                tb = __shfl_sync(0xffffffffu, tb, 0);
                if (tb + ntr > C->trail_cap) {
                    if (lane == 0) atomicExch(&C->status, CT_ERR_OOM);
                } else {
                    int off = tb;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (need[e]) {
                            const int p = off + __popc(nb[e] & lanemask_lt());
                            T.trailKey[p] = make_int2(w[e], prev[e]);
                            T.trailOld[p] = cur[e];
                            T.lastpos[w[e]] = p;
                        }
                        off += __popc(nb[e]);
                    }
                }
            }

            // Stable partition of the segment: survivors first, removed after.
            uint32_t ab[E];
            int nal = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) { ab[e] = __ballot_sync(0xffffffffu, alive[e]); nal += __popc(ab[e]); }
            if (nal != c) {
                int before = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (act[e]) {
                        const int sb = before + __popc(ab[e] & lanemask_lt());
                        const int pos = e * 32 + lane;
                        idx[alive[e] ? sb : nal + (pos - sb)] = w[e];
                    }
                    before += __popc(ab[e]);
                }
                if (lane == 0) T.segCnt[seg] = nal;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) words += __shfl_xor_sync(0xffffffffu, words, o);
            if (lane == 0) {
                atomicAdd(&s_live, (uint32_t)nal);
                atomicAdd(&s_livein, (uint32_t)c);
                atomicAdd(&s_words, words);
                atomicAdd(&s_trail, (uint32_t)ntr);
            }
        }
    }

    // Last-block-done: every thread fences its own writes before the ticket.
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&C->live, s_live);
        atomicAdd(&C->live_in, s_livein);
        atomicAdd(&C->words_in, s_words);
        if (s_trail) atomicAdd(&C->trail_added, (int)s_trail);
        __threadfence();
        const unsigned t = atomicAdd(&C->done_update, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // Algorithm 1, line 5: fail when currTable is all zero.
    if (__ldcg(&C->live) == 0u) {
        if (threadIdx.x == 0) atomicExch(&C->status, CT_INFEASIBLE);
        return;
    }
    if (__ldcg(&C->status) != CT_OK) return;

    // Residue probes for every value of s_sup (Algorithm 3 with residues).
    __shared__ int s_hits;
    if (threadIdx.x == 0) s_hits = 0;
    __syncthreads();
    const size_t W4 = (size_t)T.W4;
    int hits = 0;
    for (int r = threadIdx.x; r < T.R; r += blockDim.x) {
        const int i = T.rowVar[r];
        if (!T.varSup[i]) continue;
        const int a = r - T.varRow0[i];
        if (!((dom[domOff[i] + (a >> 5)] >> (a & 31)) & 1u)) continue;
        bool hit = false;
        if (T.useResidues) {
            const int res = T.residue[r];
            hit = nz(and4(ld_sup(T.sup + (size_t)r * W4 + res), __ldcg(T.curr + res)));
        }
        if (hit) {
            ++hits;
        } else {
            const unsigned m = atomicAdd(&C->nmiss, 1u);
            T.missRow[m] = r;
            T.foundChunk[m] = kNoChunk;
        }
    }
    if (hits) atomicAdd(&s_hits, hits);
    __syncthreads();
    if (threadIdx.x == 0) C->hits = s_hits;
}

// ---------------------------------------------------------------------------
// scan: search the live chunks for the values whose residue missed; the last
// CTA applies the result (Algorithm 3) and writes the status block.
// ---------------------------------------------------------------------------
template <int E>
__global__ void __launch_bounds__(512)
ct_scan_kernel(TableDev T, uint32_t* __restrict__ dom, const int32_t* __restrict__ domOff) {
    Ctrl* C = T.ctrl;
    const int st = C->status;
    if (st != CT_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) write_header(T, st);
        return;
    }
    __shared__ int s_last, s_pruned;

    const int lane = threadIdx.x & 31;
    const int seg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nm = (int)C->nmiss;

    if (nm > 0 && seg < T.nseg) {
        const int c = T.segCnt[seg];
        const int32_t* idx = T.idx + seg * T.S;
        bool act[E];
        int w[E];
        uint4 cur[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            act[e] = e * 32 + lane < c;
            w[e] = act[e] ? idx[e * 32 + lane] : 0;
            cur[e] = act[e] ? T.curr[w[e]] : make_uint4(0u, 0u, 0u, 0u);
        }
        if (__any_sync(0xffffffffu, act[0])) {
            const size_t W4 = (size_t)T.W4;
            constexpr int U = 4;
            for (int m0 = 0; m0 < nm; m0 += U) {
                int cand[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    cand[k] = kNoChunk;
                    if (m0 + k < nm) {
                        const uint4* row = T.sup + (size_t)T.missRow[m0 + k] * W4;
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if (act[e] && nz(and4(ld_sup(row + w[e]), cur[e]))) cand[k] = min(cand[k], w[e]);
                    }
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    if (m0 + k < nm) {
                        const int mn = __reduce_min_sync(0xffffffffu, cand[k]);
                        if (lane == 0 && mn != kNoChunk) atomicMin(&T.foundChunk[m0 + k], mn);
                    }
                }
            }
        }
    }

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(&C->done_scan, 1u);
        s_last = (t == gridDim.x - 1);
        s_pruned = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // Apply: a value with no supporting chunk leaves its domain (Algorithm 3 line 4).
    int pruned = 0;
    for (int m = threadIdx.x; m < nm; m += blockDim.x) {
        const int r = __ldcg(&T.missRow[m]);
        const int fc = __ldcg(&T.foundChunk[m]);
        if (fc != kNoChunk) {
            T.residue[r] = fc;
        } else {
            const int i = T.rowVar[r];
            const int a = r - T.varRow0[i];
            atomicAnd(&dom[domOff[i] + (a >> 5)], ~(1u << (a & 31)));
            T.changed[i] = 1;
            ++pruned;
        }
    }
    if (pruned) atomicAdd(&s_pruned, pruned);
    __syncthreads();

    // lastDom := the filtered domains (lastSizes update of Algorithm 3 line 5);
    // the same words go to the status block for the host.
    uint32_t* outDom = reinterpret_cast<uint32_t*>(T.statusBlk + kStatusHdr + T.nChangedWords);
    for (int i = threadIdx.x; i < T.arity; i += blockDim.x) {
        const int nw = T.varNW[i];
        const uint32_t* d = dom + domOff[i];
        uint32_t* l = T.lastDom + T.varLD[i];
        uint32_t* o = outDom + T.varLD[i];
        for (int q = 0; q < nw; ++q) {
            const uint32_t v = __ldcg(d + q);
            l[q] = v;
            o[q] = v;
        }
    }
    for (int q = threadIdx.x; q < T.nChangedWords; q += blockDim.x) {
        uint32_t bits = 0u;
        for (int b = 0; b < 32 && q * 32 + b < T.arity; ++b)
            if (T.changed[q * 32 + b]) bits |= 1u << b;
        T.statusBlk[kStatusHdr + q] = (int32_t)bits;
    }
    if (threadIdx.x == 0) {
        C->pruned = s_pruned;
        write_header(T, CT_OK);
        T.statusBlk[kSlotPruned] = s_pruned;
    }
}

// ---------------------------------------------------------------------------
// save / restore of backtrack levels
// ---------------------------------------------------------------------------
__global__ void ct_save_kernel(TableDev T, int level) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    int32_t* ls = T.levelSeg + (size_t)level * T.nseg;
    uint32_t* ld = T.levelDom + (size_t)level * T.DW;
    for (int s = tid; s < T.nseg; s += nth) ls[s] = T.segCnt[s];
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
    const int32_t* ls = T.levelSeg + (size_t)level * T.nseg;
    const uint32_t* ld = T.levelDom + (size_t)level * T.DW;
    for (int s = tid; s < T.nseg; s += nth) T.segCnt[s] = ls[s];
    for (int q = tid; q < T.DW; q += nth) T.lastDom[q] = ld[q];
    if (tid == 0) {
        T.ctrl->trail_top = mark;
        T.ctrl->cur_mark = newMark;
        T.ctrl->status = CT_OK;
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

}  // namespace

cudaError_t launch_plan(const TableDev& T, const uint32_t* dom, const int32_t* domOff, cudaStream_t s) {
    ct_plan_kernel<<<1, kPlanThreads, 0, s>>>(T, dom, domOff);
    return cudaGetLastError();
}

cudaError_t launch_update(const TableDev& T, int E, int wpb, const uint32_t* dom, const int32_t* domOff,
                          cudaStream_t s) {
    const int grid = (T.nseg + wpb - 1) / wpb;
    switch (E) {
        case 1: ct_update_kernel<1><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        case 2: ct_update_kernel<2><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        case 4: ct_update_kernel<4><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(const TableDev& T, int E, int wpb, uint32_t* dom, const int32_t* domOff,
                        cudaStream_t s) {
    const int grid = (T.nseg + wpb - 1) / wpb;
    switch (E) {
        case 1: ct_scan_kernel<1><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        case 2: ct_scan_kernel<2><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        case 4: ct_scan_kernel<4><<<grid, wpb * 32, 0, s>>>(T, dom, domOff); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
