// ct_model_kernels.cu -- a network of tables propagated to its fixpoint in one
// cooperative launch, the batched trail undo of several tables, and the state
// copies of the batched search's table clones.
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ct_device.cuh"

namespace ctk {

namespace {

// ---------------------------------------------------------------------------
// A network of tables to its fixpoint in one cooperative launch (Sec. 2:
// propagation removes unsupported values until GAC holds everywhere or a
// failure is found). Rounds are Jacobi steps: every table of the round's work
// list propagates on the same domains (plan, updateTable, failure test,
// filterDomains); their removals are applied together; a table joins the next
// round when another table removed a value of one of its variables. The GAC
// closure is unique, so the order of the propagations does not matter.
// ---------------------------------------------------------------------------

// The update's live/words counters are a table's control block from `live` on.
static_assert(offsetof(Ctrl, live_in) == offsetof(Ctrl, live) + 4 * kCntLiveIn &&
                  offsetof(Ctrl, words_in) == offsetof(Ctrl, live) + 4 * kCntWords && kCntLive == 0,
              "counter block layout");

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

// The same search by one lane for its own u (binary search: the lanes of a
// warp look up different units at once).
__device__ __forceinline__ int lane_find_prefix(const int32_t* pre, int n, int u, bool global) {
    int lo = 0, hi = n - 1;  // pre[lo] <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre_at(pre, mid, global) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Exclusive prefixes of the segments and of the supports rows of work[k] over
// k < n into unitOut[0..n] and rowOut[0..n] (one CTA): each thread sums a run
// of entries, warps scan by shuffles, warp totals go through shared memory.
__device__ void work_prefix(const ModelDev& M, const int32_t* work, int n, int32_t* unitOut, int32_t* rowOut,
                            Smem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kThreads - 1) / kThreads;
    const int b0 = tid * per, b1 = min(n, b0 + per);
    // the run's tables eight at a time, their loads issued together
    constexpr int kB = 8;
    int su = 0, sr = 0;
    for (int k0 = b0; k0 < b1; k0 += kB) {
        int t[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) t[u] = k0 + u < b1 ? __ldcg(&work[k0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (t[u] >= 0) {
                su += M.tabs[t[u]].nseg;
                sr += M.tabs[t[u]].R;
            }
    }
    int iu = su, ir = sr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, iu, o);
        const int c = __shfl_up_sync(0xffffffffu, ir, o);
        if (lane >= o) {
            iu += a;
            ir += c;
        }
    }
    if (lane == 31) {
        sm.scan[warp] = iu;
        sm.scan[kWarps + warp] = ir;
    }
    __syncthreads();
    int ru = iu - su, rr = ir - sr, tu = 0, tr = 0;
    for (int w = 0; w < kWarps; ++w) {
        const int wu = sm.scan[w], wr = sm.scan[kWarps + w];
        if (w < warp) {
            ru += wu;
            rr += wr;
        }
        tu += wu;
        tr += wr;
    }
    for (int k0 = b0; k0 < b1; k0 += kB) {
        int t[kB], ns[kB], nr[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) t[u] = k0 + u < b1 ? __ldcg(&work[k0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            ns[u] = t[u] >= 0 ? M.tabs[t[u]].nseg : 0;
            nr[u] = t[u] >= 0 ? M.tabs[t[u]].R : 0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (t[u] >= 0) {
                unitOut[k0 + u] = ru;
                rowOut[k0 + u] = rr;
                ru += ns[u];
                rr += nr[u];
            }
    }
    if (tid == 0) {
        unitOut[n] = tu;
        rowOut[n] = tr;
    }
    __syncthreads();
}

// Algorithm 1 lines 1-3 and the row list of Algorithm 2 for a table with
// warpPlan set, by one warp (lane i holds variable i and its domain words in
// registers): the outputs of plan() in global mode (row counts and delta
// flags, first code of each variable, s_sup, row codes in variable order,
// each variable's last code marked) and the table's call counters. A domain
// that grew since the table's last propagation is a state error; an empty one
// fails the table's node.
__device__ void plan_warp(const ModelDev& M, const TableDev& T, const VarLayout& V, int t) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const bool own = lane < T.arity;
    uint32_t d[kWarpPlanWords], l[kWarpPlanWords];
    int nw = 0, nd = 0, ndel = 0;
    uint32_t grow = 0u;
    if (own) {
        nw = V.nw(lane);
        const uint32_t* dp = M.dom + V.off(lane);
        const uint32_t* lp = T.lastDom + V.ld(lane);
#pragma unroll
        for (int q = 0; q < kWarpPlanWords; ++q) {
            d[q] = q < nw ? __ldcg(dp + q) : 0u;
            l[q] = q < nw ? __ldcg(lp + q) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kWarpPlanWords; ++q) {
            grow |= d[q] & ~l[q];
            nd += __popc(d[q]);
            ndel += __popc(l[q] & ~d[q]);
        }
    }
    // Algorithm 2, line 3: the delta mask when |Delta| < |dom| (strict)
    const bool delta = ndel > 0 && ndel < nd;
    const int k = ndel > 0 ? (delta ? ndel : nd) : 0;
    const bool bad = __ballot_sync(FULL, grow != 0u) != 0u;
    const bool empty = __ballot_sync(FULL, own && nd == 0) != 0u;
    const int nval = __popc(__ballot_sync(FULL, ndel > 0));
    const int ndelta = __popc(__ballot_sync(FULL, delta));
    const int nsup = __popc(__ballot_sync(FULL, nd > 1));
    if (own) {
        T.planK[lane] = delta ? (k | kCodeDelta) : k;
        T.varSup[lane] = nd > 1;
    }
    int rows = (bad || empty) ? 0 : k;
    int incl = rows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += a;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (own) T.planRowOff[lane] = incl - rows;
    if (rows > 0) {
        const int row0 = V.row0(lane);
        int out = incl - rows;
        const int last = incl - 1;
#pragma unroll
        for (int q = 0; q < kWarpPlanWords; ++q) {
            uint32_t bits = delta ? (l[q] & ~d[q]) : d[q];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                int code = row0 + q * 32 + b;
                if (delta) code |= kCodeDelta;
                if (out == last) code |= kCodeLast;
                T.codes[out++] = code;
            }
        }
    }
    if (lane == 0) {
        Ctrl* Tc = T.ctrl;
        Tc->nrows = total;
        Tc->nval = nval;
        Tc->ndelta = ndelta;
        Tc->nreset = nval - ndelta;
        Tc->nsup = nsup;
        if (bad) atomicCAS(&M.ctrl->status, CT_OK, CT_ERR_STATE);
        else if (empty) M.nodeStatus[t / M.nodeTables] = CT_INFEASIBLE;
    }
}

// Value r of table t has no support: clear it from the shared domains and, for
// a positive table, from the table's lastDom (no valid tuple carries it), and
// mark its variable as pruned by t (-2: by several tables). A negative table's
// removed value still has valid forbidden tuples, which its next pass removes
// as Delta, and that pass is due: one pass of a negative table is not GAC for
// it (a removal shrinks the products the other values are compared with), so
// its own removals schedule it again (-2).
__device__ __forceinline__ void remove_value(const ModelDev& M, const TableDev& T, int t, int r, int32_t* pruned) {
    const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
    const int i = T.rowVar[r];
    const int a = r - V.row0(i);
    atomicAnd(&M.dom[V.off(i) + (a >> 5)], ~(1u << (a & 31)));
    const int v = M.scopeVar[M.scopeBase[t] + i];
    if (T.negative) {
        atomicExch(&pruned[v], -2);
        return;
    }
    atomicAnd(&T.lastDom[V.ld(i) + (a >> 5)], ~(1u << (a & 31)));
    const int old = atomicCAS(&pruned[v], -1, t);
    if (old != -1 && old != t) atomicExch(&pruned[v], -2);
}

// ---------------------------------------------------------------------------
// The batched search on the device (search mode). Between two rounds of the
// fixpoint, one warp per slot decides: a slot whose node is at its fixpoint
// (no table of it in the next round) or failed branches on the first-fail
// variable (left: x = min D(x)), backtracks to the deepest frame whose right
// branch (x != min) is untried, or, with its subtree done, takes the next
// open node from the device queue. Restores are queued and done by the whole
// grid after a barrier: a table's trail entries above the level's mark are
// undone (each chunk written once), its non-zero index comes from the level's
// snapshot, and its last-seen domains from the level's domains (a level is
// saved at a fixpoint, where every table has seen the domains of its scope).
// ---------------------------------------------------------------------------
constexpr unsigned FULLM = 0xffffffffu;

__device__ __forceinline__ size_t lvl(const SearchDev& S, int s, int L) {
    return (size_t)s * (S.maxLevels + 1) + L;
}

// Append table k (model index) of slot s for each k in list[0..n) to the next
// round's work list (warp-aggregated).
__device__ void append_tables(const SearchDev& S, int s, const int32_t* list, int n, int32_t* next, int32_t* nnext) {
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool ok = i < n;
        const unsigned bal = __ballot_sync(FULLM, ok);
        int base = 0;
        if (lane == 0) base = atomicAdd(nnext, __popc(bal));
        base = __shfl_sync(FULLM, base, 0);
        if (ok) next[base + __popc(bal & lanemask_lt())] = s * S.T + (list ? list[i] : i);
    }
}

// First-fail over the slot's domains: the unfixed variable with the smallest
// domain, ties to the lowest index; -1 when every variable is fixed (warp-wide).
__device__ int warp_first_fail(const SearchDev& S, const uint32_t* dom) {
    const int lane = threadIdx.x & 31;
    int best = 0x7fffffff, bx = -1;
    for (int v = lane; v < S.nv; v += 32) {
        int sz = 0;
        const int o = S.varOff[v], nw = S.varNW[v];
        for (int q = 0; q < nw; ++q) sz += __popc(__ldcg(dom + o + q));
        if (sz > 1 && sz < best) {
            best = sz;
            bx = v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int ob = __shfl_xor_sync(FULLM, best, o), ox = __shfl_xor_sync(FULLM, bx, o);
        if (ob < best || (ob == best && ox >= 0 && (bx < 0 || ox < bx))) {
            best = ob;
            bx = ox;
        }
    }
    return bx;
}

__device__ int min_value_dev(const SearchDev& S, const uint32_t* dom, int x) {
    for (int q = 0; q < S.varNW[x]; ++q) {
        const uint32_t w = __ldcg(dom + S.varOff[x] + q);
        if (w) return q * 32 + __ffs(w) - 1;
    }
    return 0;
}

// Level L of slot s holds the current state: domains, each table's trail mark,
// live count and non-zero index; the tables' calls trail from that mark on.
__device__ void save_level(const ModelDev& M, const SearchDev& S, int s, int L) {
    const int lane = threadIdx.x & 31;
    const uint32_t* dom = M.dom + (size_t)s * S.DWs;
    uint32_t* ld = S.levelDom + lvl(S, s, L) * S.DWs;
    for (int q = lane; q < S.DWs; q += 32) ld[q] = __ldcg(dom + q);
    for (int k = lane; k < S.T; k += 32) {
        const int j = s * S.T + k;
        const Ctrl* c = M.tabs[j].ctrl;
        const int top = __ldcg(&c->trail_top);
        S.markAt[lvl(S, s, L) * S.T + k] = top;
        S.liveAt[lvl(S, s, L) * S.T + k] = __ldcg(&c->live_state);
        S.calls[j].mark = top;
    }
    // the index masks of all the slot's tables, word by word over the lanes,
    // four loads in flight per lane
    uint32_t* snap = S.snapSeg + lvl(S, s, L) * S.segTotal;
    for (int i0 = lane; i0 < S.segTotal; i0 += 128) {
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + 32 * u;
            v[u] = 0u;
            if (i < S.segTotal) {
                const int k = __ldg(&S.segTabOf[i]);
                v[u] = __ldcg(S.segPtr[s * S.T + k] + (i - __ldg(&S.segOff[k])));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + 32 * u < S.segTotal) snap[i0 + 32 * u] = v[u];
    }
}

// Queue the restore of every table of slot s to level L; their calls trail
// from that level's marks again.
__device__ void queue_restore(const SearchDev& S, int s, int L) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(&S.ctr->nrestQ, S.T);
    base = __shfl_sync(FULLM, base, 0);
    // (at most one restore per slot and decision phase: the queue holds B * T)
    for (int k = lane; k < S.T; k += 32) {
        S.restQ[base + k] = make_int4(s * S.T + k, L, 0, 0);
        S.calls[s * S.T + k].mark = S.markAt[lvl(S, s, L) * S.T + k];
    }
}

// A node is issued (counted) unless the node limit is reached.
__device__ bool issue_node(const SearchDev& S, int depth) {
    const int lane = threadIdx.x & 31;
    unsigned long long o = 0;
    if (lane == 0) {
        o = atomicAdd(&S.ctr->nodes, 1ull);
        if (S.nodeLimit <= 0 || (long long)o < S.nodeLimit) atomicMax(&S.ctr->maxDepth, depth);
    }
    o = __shfl_sync(FULLM, o, 0);
    return S.nodeLimit <= 0 || (long long)o < S.nodeLimit;
}

// The tables of variable x of slot s go to the next round; a variable in no
// table still takes one round (table 0 of the slot, which finds nothing to
// do), so that every issued node is decided after a round and every queued
// restore is done before the slot saves a level again.
__device__ void append_var(const SearchDev& S, int s, int x, int32_t* next, int32_t* nnext) {
    const int t0 = S.varTabStart[x], t1 = S.varTabStart[x + 1];
    if (t1 > t0) {
        append_tables(S, s, S.varTabList + t0, t1 - t0, next, nnext);
    } else {
        const int32_t zero = 0;
        append_tables(S, s, &zero, 1, next, nnext);
    }
}

// One warp: move slot s on when its node is done. Returns after issuing a
// node (its tables are in the next round) or with the slot idle; at most one
// restore of the slot is queued.
__device__ void decide_slot(const ModelDev& M, const SearchDev& S, int s, int32_t* next, int32_t* nnext) {
    const int lane = threadIdx.x & 31;
    uint32_t* dom = M.dom + (size_t)s * S.DWs;
    for (int guard = 0; guard < 2; ++guard) {
        if (!S.active[s]) {
            // an idle slot takes the next open node (its tables back at level 0, the root)
            if (__ldcg(&S.ctr->error) != CT_OK) return;
            int o = 0;
            if (lane == 0) o = atomicAdd(&S.ctr->nextOpen, 1);
            o = __shfl_sync(FULLM, o, 0);
            if (o >= S.nopen) return;
            if (!issue_node(S, S.openDepth[o])) return;
            queue_restore(S, s, 0);
            for (int q = lane; q < S.DWs; q += 32) dom[q] = S.openDom[(size_t)o * S.DWs + q];
            if (lane == 0) {
                S.active[s] = 1;
                S.depth[s] = 0;
                S.openIdx[s] = o;
                S.depth0[s] = S.openDepth[o];
                S.busy[s] = 0;
                M.nodeStatus[s] = CT_OK;
            }
            append_tables(S, s, nullptr, S.T, next, nnext);
            return;
        }
        if (__ldcg(&S.busy[s])) {  // its node is still propagating
            if (lane == 0) S.busy[s] = 0;
            return;
        }
        const bool failed = __ldcg(&M.nodeStatus[s]) != CT_OK;
        if (lane == 0) M.nodeStatus[s] = CT_OK;
        int d = S.depth[s];
        if (!failed) {
            const int x = warp_first_fail(S, dom);
            if (x >= 0) {
                // left branch x = min D(x), after saving level d + 1
                if (d >= S.maxLevels) {
                    if (lane == 0) atomicCAS(&S.ctr->error, CT_OK, CT_ERR_LEVEL);
                    if (lane == 0) S.active[s] = 0;
                    return;
                }
                if (!issue_node(S, S.depth0[s] + d + 1)) {
                    if (lane == 0) S.active[s] = 0;
                    return;
                }
                const int a = min_value_dev(S, dom, x);
                save_level(M, S, s, d + 1);
                __syncwarp();
                for (int q = lane; q < S.varNW[x]; q += 32) dom[S.varOff[x] + q] = q == (a >> 5) ? 1u << (a & 31) : 0u;
                if (lane == 0) {
                    S.frames[(size_t)s * S.maxLevels + d] = make_int4(x, a, 0, 0);
                    S.depth[s] = d + 1;
                }
                append_var(S, s, x, next, nnext);
                return;
            }
            // every variable fixed: a solution. A slot takes open nodes in
            // increasing (depth-first) order and searches each subtree
            // depth-first, so its first solution is the first of its subtrees;
            // it is kept for the host.
            bool first = false;
            if (lane == 0) {
                atomicAdd(&S.ctr->solutions, 1ull);
                first = S.openIdx[s] < S.firstOpen[s];
                if (first) S.firstOpen[s] = S.openIdx[s];
            }
            first = __shfl_sync(FULLM, first, 0);
            if (first)
                for (int q = lane; q < S.DWs; q += 32) S.firstSol[(size_t)s * S.DWs + q] = __ldcg(dom + q);
        } else if (lane == 0) {
            atomicAdd(&S.ctr->fails, 1ull);
        }
        // backtrack: the deepest frame with an untried right branch
        while (d > 0 && S.frames[(size_t)s * S.maxLevels + d - 1].z != 0) --d;
        if (d == 0) {
            if (lane == 0) {
                S.depth[s] = 0;
                S.active[s] = 0;
            }
            __syncwarp();
            continue;  // the subtree is done: take the next open node
        }
        const int4 f = S.frames[(size_t)s * S.maxLevels + d - 1];
        if (!issue_node(S, S.depth0[s] + d)) {
            if (lane == 0) S.active[s] = 0;
            return;
        }
        queue_restore(S, s, d);
        const uint32_t* ld = S.levelDom + lvl(S, s, d) * S.DWs;
        for (int q = lane; q < S.DWs; q += 32) dom[q] = ld[q];
        __syncwarp();
        if (lane == 0) {
            dom[S.varOff[f.x] + (f.y >> 5)] &= ~(1u << (f.y & 31));
            S.frames[(size_t)s * S.maxLevels + d - 1] = make_int4(f.x, f.y, 1, 0);
            S.depth[s] = d;
        }
        append_var(S, s, f.x, next, nnext);
        return;
    }
}

// One warp per queued restore: table j back to level L of its slot.
__device__ void restore_table(const ModelDev& M, const SearchDev& S, int j, int L) {
    const int lane = threadIdx.x & 31;
    const int s = j / S.T, k = j - s * S.T;
    const TableDev& T = M.tabs[j];
    // (the decision phase ran on other CTAs: its records are read through L2)
    const int mark = __ldcg(&S.markAt[lvl(S, s, L) * S.T + k]);
    const int top = __ldcg(&T.ctrl->trail_top);
    for (int p0 = mark + lane; p0 < top; p0 += 128) {  // four entries in flight per lane
        int2 key[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + 32 * u;
            key[u] = p < top ? __ldcg(&T.trailKey[p]) : make_int2(-1, 0x7fffffff);
        }
        uint4 old[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (key[u].y < mark) old[u] = __ldcg(&T.trailOld[p0 + 32 * u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (key[u].y < mark) {
                T.curr[key[u].x] = old[u];
                T.lastpos[key[u].x] = key[u].y;
            }
        }
    }
    const uint32_t* snap = S.snapSeg + lvl(S, s, L) * S.segTotal + S.segOff[k];
    for (int q = lane; q < T.nseg; q += 32) T.segMask[q] = __ldcg(snap + q);
    // last-seen domains: the level's domains of the table's scope
    const uint32_t* ld = S.levelDom + lvl(S, s, L) * S.DWs;
    const int b0 = M.scopeBase[j];
    for (int i = lane; i < T.arity; i += 32) {
        const VarLayout V(T, nullptr, M.scopeOff + b0);
        const int o = V.off(i) - s * S.DWs;
        for (int q = 0; q < V.nw(i); ++q) T.lastDom[V.ld(i) + q] = __ldcg(ld + o + q);
    }
    __syncwarp();
    if (lane == 0) {
        T.ctrl->trail_top = mark;
        T.ctrl->live_state = __ldcg(&S.liveAt[lvl(S, s, L) * S.T + k]);
        T.ctrl->status = CT_OK;
    }
}

template <int U, bool kSearch, int kMinBlocks = 2>
__global__ void __launch_bounds__(kThreads, kMinBlocks) ct_model_kernel(const __grid_constant__ ModelDev M) {
    __shared__ Smem sm;
    ModelCtrl* C = M.ctrl;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    int32_t* preU = sm.codes;                               // unit prefix of the round (smem copy)
    int32_t* preR = reinterpret_cast<int32_t*>(sm.dom);     // row prefix of the round (smem copy)
    GridBarrier bar;
    bar_init(bar, &C->bar_count, &C->bar_base, &C->status, M.spinLimit ? M.spinLimit : kBarrierSpinLimit);
    auto sync = [&]() { return bar_sync(bar, &sm.flag[0]) != 0; };
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
    int cur = 0, round = 0, launchRounds = 0;
    // search mode: the search state, and its step between two rounds (the
    // decisions, a barrier, the queued restores, a barrier)
    SearchDev Sd{};
    if (kSearch) Sd = *M.search;
    auto search_step = [&]() -> bool {
        int32_t* nl = M.work + (size_t)cur * M.ntables;
        int32_t* nc = &C->nnext[round & 1];
        for (int s = gwarp; s < Sd.B; s += nwarps) decide_slot(M, Sd, s, nl, nc);
        if (!sync()) return false;
        const int nr = __ldcg(&Sd.ctr->nrestQ);
        for (int q = gwarp; q < nr; q += nwarps) {
            const int4 e = __ldcg(&Sd.restQ[q]);
            restore_table(M, Sd, e.x, e.y);
        }
        if (!sync()) return false;
        if (blockIdx.x == 0 && tid == 0) Sd.ctr->nrestQ = 0;  // read by no CTA before the next decisions
        return true;
    };
    if (kSearch) {
        cur = __ldcg(&Sd.ctr->cur);
        round = __ldcg(&Sd.ctr->round);
        if (!__ldcg(&Sd.ctr->started)) {
            if (!search_step()) return;
            if (blockIdx.x == 0 && tid == 0) Sd.ctr->started = 1;
        }
    }
    for (;;) {
        const int nwork = kSearch ? __ldcg(&C->nnext[round & 1])
                                  : round > 0 ? __ldcg(&C->nnext[round & 1]) : M.nworkIn ? __ldcg(M.nworkIn) : __ldcg(&C->nwork);
        if (kSearch && nwork == 0) {
            // every slot idle, no open node left (or the node limit reached)
            if (blockIdx.x == 0 && tid == 0) Sd.ctr->done = 1;
            break;
        }
        phase(round == 0 ? 0 : 6);
        const int32_t* work = M.work + (size_t)cur * M.ntables;
        int32_t* pruned = M.prunedBy + (size_t)(round & 1) * M.nvars;       // written by this round
        int32_t* prunedNext = M.prunedBy + (size_t)((round + 1) & 1) * M.nvars;
        // the collector of the next round's tables was last read two rounds ago,
        // and so was the other miss counter
        if (blockIdx.x == 0 && tid == 0) {
            C->nnext[(round + 1) & 1] = 0;
            C->nmiss[(round + 1) & 1] = 0;
            C->nscanAll[(round + 1) & 1] = 0;
        }

        // plan (Algorithm 1 lines 1-3): one warp per small table (warpPlan), by
        // the warps of every CTA but the last, which computes the round's
        // prefixes; one CTA per other table
        {
            const int planCtas = gridDim.x > 1 ? gridDim.x - 1 : 1;
            if (blockIdx.x < planCtas) {
                for (int k = gwarp; k < nwork; k += planCtas * kWarps) {
                    const int t = __ldcg(&work[k]);
                    const TableDev& T = M.tabs[t];
                    if (!T.warpPlan) continue;
                    const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
                    // the pending level snapshot, as in the CTA path below
                    const int sf = __ldcg(&M.calls[t].snapFrom), stp = __ldcg(&M.calls[t].snapTo);
                    if (sf < stp && __ldcg(&M.snapTaken[t]) == 0) {
                        const size_t l = (size_t)sf;
                        for (int q = lane; q < T.nseg; q += 32) T.levelSeg[l * T.nseg + q] = __ldcg(&T.segMask[q]);
                        for (int q = lane; q < T.DW; q += 32) T.levelDom[l * T.DW + q] = __ldcg(&T.lastDom[q]);
                        __syncwarp();
                        if (lane == 0) M.snapTaken[t] = 1;
                    }
                    __syncwarp();  // the snapshot reads lastDom before the plan's loads of it
                    plan_warp(M, T, V, t);
                }
            }
        }
        // the CTA's share of the work list (entries blockIdx.x + j * gridDim.x),
        // 256 entries tested at once (one per thread); the tables without a
        // warp plan are planned one after the other by the whole CTA
        // (sm.codes is free until the round's prefixes are staged)
        for (int k0 = blockIdx.x; k0 < nwork; k0 += gridDim.x * kThreads) {
            const int kt = k0 + tid * gridDim.x;
            const bool need = kt < nwork && !M.tabs[__ldcg(&work[kt])].warpPlan;
            sm.codes[tid] = need ? kt : -1;
            if (!__syncthreads_or(need)) continue;
            for (int j = 0; j < kThreads; ++j) {
                const int k = sm.codes[j];
                if (k < 0) continue;  // the same for every thread of the CTA
                const int t = __ldcg(&work[k]);
                const TableDev& T = M.tabs[t];
                const VarLayout V(T, nullptr, M.scopeOff + M.scopeBase[t]);
                // Levels saved since the table's last propagation all hold its state
                // as it is now: one snapshot, in the lowest one's slot, taken before
                // this launch first changes the table (a table this launch does not
                // propagate keeps them pending).
                ModelTabCall cl;
                cl.mark = __ldcg(&M.calls[t].mark);
                cl.snapFrom = __ldcg(&M.calls[t].snapFrom);
                cl.snapTo = __ldcg(&M.calls[t].snapTo);
                if (cl.snapFrom < cl.snapTo && __ldcg(&M.snapTaken[t]) == 0) {
                    const size_t l = (size_t)cl.snapFrom;
                    for (int q = tid; q < T.nseg; q += kThreads) T.levelSeg[l * T.nseg + q] = __ldcg(&T.segMask[q]);
                    for (int q = tid; q < T.DW; q += kThreads) T.levelDom[l * T.DW + q] = __ldcg(&T.lastDom[q]);
                    if (tid == 0) M.snapTaken[t] = 1;
                }
                plan(T, V, M.dom, T.planK, T.planRowOff, T.varSup, T.codes, nullptr, sm);
                if (T.negative && tid == 0 && !sm.flags[0] && !sm.flags[1]) {
                    // a value of x_i loses its support when its valid forbidden
                    // tuples are all prod_{j != i} |D_j| combinations: the products,
                    // saturated at 2^62
                    const unsigned long long cap = 1ull << 62;
                    auto mul = [&](unsigned long long x, unsigned long long y) {
                        return (y != 0 && x > cap / y) ? cap : x * y;
                    };
                    unsigned long long pre = 1ull;
                    for (int i = 0; i < T.arity; ++i) {
                        T.other[i] = pre;
                        pre = mul(pre, (unsigned long long)sm.nd[i]);
                    }
                    unsigned long long suf = 1ull;
                    for (int i = T.arity - 1; i >= 0; --i) {
                        T.other[i] = mul(T.other[i], suf);
                        suf = mul(suf, (unsigned long long)sm.nd[i]);
                    }
                }
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
            __syncthreads();  // sm.codes is rewritten by the next stride
        }
        // the prefixes by the last CTA, which plans no table when the work
        // list is shorter than the grid
        if (blockIdx.x == gridDim.x - 1) work_prefix(M, work, nwork, M.unitPrefix, M.rowPrefix, sm);
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

        // updateTable (Algorithm 2) over (table, segment) units, unit u to warp
        // u % nwarps (a crowded table's segments spread over the grid). A warp
        // looks up the tables of its next 32 units at once (one lane each:
        // work-list entry, row count, mark), and loads the next unit's segment
        // state while the current unit's rows are read.
        for (int ub = gwarp; ub < totalUnits; ub += 32 * nwarps) {
            const int ul = ub + lane * nwarps;
            int lt = 0, lseg = 0, lrows = 0, lmark = -1, lneg = 0;
            if (ul < totalUnits) {
                const int k = lane_find_prefix(pU, nwork, ul, gpre);
                lt = __ldcg(&work[k]);
                lseg = ul - pre_at(pU, k, gpre);
                lrows = __ldcg(&M.tabs[lt].ctrl->nrows);
                lmark = __ldcg(&M.calls[lt].mark);
                lneg = M.tabs[lt].negative;
            }
            // a negative table goes through even with no row to OR: its
            // filter compares counts with the valid tuples left
            const bool lwork = ul < totalUnits && (lrows > 0 || lneg);
            const unsigned todo = __ballot_sync(0xffffffffu, lwork);
            SegState next;
            next.mask = 0u;
            int j = todo ? __ffs(todo) - 1 : 32;
            if (j < 32) {
                const int t0 = __shfl_sync(0xffffffffu, lt, j);
                next = load_segment(M.tabs[t0], __shfl_sync(0xffffffffu, lseg, j),
                                    __shfl_sync(0xffffffffu, lmark, j));
            }
            while (j < 32) {
                const int t = __shfl_sync(0xffffffffu, lt, j);
                const int seg = __shfl_sync(0xffffffffu, lseg, j);
                const int nrows = __shfl_sync(0xffffffffu, lrows, j);
                const int mark = __shfl_sync(0xffffffffu, lmark, j);
                const SegState S = next;
                const unsigned rest = todo & ~((2u << j) - 1u);
                const int jn = rest ? __ffs(rest) - 1 : 32;
                if (jn < 32) {
                    const int tn = __shfl_sync(0xffffffffu, lt, jn);
                    next = load_segment(M.tabs[tn], __shfl_sync(0xffffffffu, lseg, jn),
                                        __shfl_sync(0xffffffffu, lmark, jn));
                }
                const TableDev& T = M.tabs[t];
                TrailItem it;
                update_segment<U, true>(T, mark, 0, 0, seg, S, nrows, nullptr,
                                        reinterpret_cast<uint32_t*>(&T.ctrl->live), &T.ctrl->tuples, it);
                trail_warp(T, it, __ldcg(&T.ctrl->trail_cap), &C->status);
                j = jn;
            }
        }
        if (!sync()) return;
        phase(2);

        if (__ldcg(&C->status) != CT_OK) break;
        // Algorithm 1 line 5: a table whose currTable became zero fails its node
        // (a negative table with no valid forbidden tuple forbids nothing);
        // the node's tables leave the work list from the next round on.
        for (int k = blockIdx.x * kThreads + tid; k < nwork; k += gridDim.x * kThreads) {
            const int t = __ldcg(&work[k]);
            const TableDev& T = M.tabs[t];
            if (!T.negative && __ldcg(&T.ctrl->nrows) > 0 && __ldcg(&T.ctrl->live) == 0u)
                M.nodeStatus[t / M.nodeTables] = CT_INFEASIBLE;
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
        // one unit per lane; the misses are queued for the whole grid (after a
        // barrier, one warp per miss searches the live chunks after the
        // residue), and what misses there too goes to the full scan.
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
                // the residue and its two chunks are loaded before the presence
                // test (a residue is always a valid chunk): the test's own loads
                // (the row's variable, its domain offset and word) go alongside
                const bool spec = T.useResidues && !T.negative;
                uint4 sv = make_uint4(0u, 0u, 0u, 0u), cv = sv;
                if (spec) {
                    res = __ldcg(&T.residue[r]);
                    sv = ld_sup(T.sup + (size_t)r * T.W4 + res);
                    cv = __ldcg(T.curr + res);
                }
                const int i = __ldg(&T.rowVar[r]);
                const int a = r - V.row0(i);
                const bool inDom = (__ldcg(&M.dom[V.off(i) + (a >> 5)]) >> (a & 31)) & 1u;
                if (T.negative) {
                    // counted by the full scan unless the valid forbidden tuples
                    // are fewer than the value's combinations (a support then exists)
                    if (inDom && __ldcg(&T.other[i]) <= (unsigned long long)__ldcg(&T.ctrl->tuples)) {
                        const unsigned m = atomicAdd(&T.ctrl->nhard, 1u);
                        T.hardRow[m] = r;
                        T.foundChunk[m] = 0;
                        atomicAdd(&T.ctrl->nscan, 1);
                        atomicAdd(&C->nscanAll[round & 1], 1);
                    }
                } else if (__ldcg(&T.varSup[i]) && inDom) {
                    if (spec) hit = nz(and4(sv, cv));
                    need = !hit;
                }
            }
            const unsigned miss = __ballot_sync(0xffffffffu, need);
            const int nhit = __popc(__ballot_sync(0xffffffffu, hit));
            if (lane == 0 && nhit) atomicAdd(&sm.cnt[kCntHits], (unsigned)nhit);
            if (miss) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&C->nmiss[round & 1], __popc(miss));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (need) M.missQ[base + __popc(miss & lanemask_lt())] = make_int4(t, r, res, 0);
            }
        }
        if (!sync()) return;
        // One warp per queued miss. A value left without support after every
        // live chunk was tested is removed here; the undecided ones go to the
        // hard lists for the full scan. Rounds without a miss skip the probe
        // phase's barrier, rounds without a scan the scan and removal phases.
        const int nm = __ldcg(&C->nmiss[round & 1]);
        for (int q = gwarp; q < nm; q += nwarps) {
            const int4 e = __ldcg(&M.missQ[q]);
            const TableDev& T = M.tabs[e.x];
            const int o = probe_windows<true, kModelProbes>(T, e.y, e.z, sm.cnt);
            if (o != kProbeFound && lane == 0) {
                if (o == kProbeGone) {
                    remove_value(M, T, e.x, e.y, pruned);
                } else {
                    const unsigned m = atomicAdd(&T.ctrl->nhard, 1u);
                    T.hardRow[m] = e.y;
                    T.foundChunk[m] = kNoChunk;
                    atomicAdd(&T.ctrl->nscan, 1);
                    atomicAdd(&sm.cnt[kCntMiss], 1u);
                    atomicAdd(&C->nscanAll[round & 1], 1);
                }
            }
        }
        if (nm > 0 && !sync()) return;
        phase(3);

        // (no write to nscanAll after the last barrier: every CTA reads the same count)
        if (__ldcg(&C->nscanAll[round & 1]) > 0) {
            // full scans of the values whose residues and windows missed, and
            // the counts of a negative table's values
            for (int u = gwarp; u < totalUnits; u += nwarps) {
                const int k = find_prefix(pU, nwork, u, gpre);
                const TableDev& T = M.tabs[__ldcg(&work[k])];
                if (__ldcg(&T.ctrl->nscan) == 0) continue;
                if (T.negative) count_segment(T, u - pre_at(pU, k, gpre), (int)__ldcg(&T.ctrl->nhard), nullptr);
                else scan_segment<U, true>(T, u - pre_at(pU, k, gpre), (int)__ldcg(&T.ctrl->nhard), nullptr);
            }
            if (!sync()) return;
            phase(4);

            // Algorithm 3 line 4: remove the values no live tuple carries
            for (int k = blockIdx.x; k < nwork; k += gridDim.x) {
                const int t = __ldcg(&work[k]);
                const TableDev& T = M.tabs[t];
                const int nh = (int)__ldcg(&T.ctrl->nhard);
                for (int m = tid; m < nh; m += kThreads) {
                    const int r = __ldcg(&T.hardRow[m]);
                    const int fc = __ldcg(&T.foundChunk[m]);
                    if (T.negative) {
                        // fc: the value's valid forbidden tuples
                        if ((unsigned long long)(unsigned)fc >= __ldcg(&T.other[T.rowVar[r]]))
                            remove_value(M, T, t, r, pruned);
                    } else if (fc >= 0 && fc != kNoChunk) {
                        T.residue[r] = fc;
                    } else {
                        remove_value(M, T, t, r, pruned);
                    }
                }
            }
            if (!sync()) return;
            phase(5);
        }
        __syncthreads();
        if (tid == 0) {
            if (sm.cnt[kCntHits]) atomicAdd(&C->hits, sm.cnt[kCntHits]);
            if (sm.cnt[kCntLocal]) atomicAdd(&C->local, sm.cnt[kCntLocal]);
            if (sm.cnt[kCntMiss]) atomicAdd(&C->hard, sm.cnt[kCntMiss]);
            if (sm.cnt[kCntWin]) atomicAdd(&C->windows, sm.cnt[kCntWin]);
            sm.cnt[kCntHits] = sm.cnt[kCntLocal] = sm.cnt[kCntMiss] = sm.cnt[kCntWin] = 0u;
        }

        // next round (whole grid): every table of a live node that shares a
        // variable another table pruned; the other parity's marks are cleared
        // for the round after
        {
            int32_t* next = M.work + (size_t)(cur ^ 1) * M.ntables;
            int32_t* nnext = &C->nnext[(round + 1) & 1];
            const int gtid = blockIdx.x * kThreads + tid, gth = gridDim.x * kThreads;
            for (int k = gtid; k < nwork; k += gth) {
                Ctrl* Tc = M.tabs[__ldcg(&work[k])].ctrl;
                const int nr = __ldcg(&Tc->nrows);
                const unsigned long long live = nr > 0 ? __ldcg(&Tc->live) : (unsigned long long)__ldcg(&Tc->live_state);
                if (nr > 0) {
                    Tc->live_state = (int32_t)live;
                    atomicAdd(&C->bytesUpdate, 4ull * __ldcg(&Tc->words_in) * (unsigned long long)(nr + 2));
                }
                const unsigned ns = (unsigned)__ldcg(&Tc->nscan);
                if (ns) atomicAdd(&C->bytesFilter, 16ull * ns * live);
                Tc->live = 0u; Tc->live_in = 0u; Tc->words_in = 0u; Tc->nhard = 0u; Tc->nrows = 0; Tc->nscan = 0;
                Tc->tuples = 0u;
            }
            for (int t0 = gtid - lane; t0 < M.ntables; t0 += gth) {  // warp-uniform trip count
                const int t = t0 + lane;
                bool dirty = false;
                if (t < M.ntables) {
                    // scope variables eight at a time, their marks loaded together
                    const bool alive = __ldcg(&M.nodeStatus[t / M.nodeTables]) == CT_OK;
                    const int j1 = M.scopeBase[t + 1];
                    for (int j = M.scopeBase[t]; j < j1; j += 8) {
                        int v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) v[u] = j + u < j1 ? M.scopeVar[j + u] : -1;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int p = v[u] >= 0 ? __ldcg(&pruned[v[u]]) : -1;
                            dirty |= p != -1 && p != t;
                        }
                    }
                    dirty &= alive;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, dirty);
                if (bal) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(nnext, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (dirty) next[base + __popc(bal & lanemask_lt())] = t;
                }
                if (kSearch && dirty) Sd.busy[t / M.nodeTables] = 1;  // its node goes on next round
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
        if (kSearch) {
            if (!search_step()) return;
            if (++launchRounds >= Sd.roundBudget) {
                // the launch's share of rounds is spent: the host launches again
                if (blockIdx.x == 0 && tid == 0) {
                    Sd.ctr->cur = cur;
                    Sd.ctr->round = round;
                }
                break;
            }
            continue;
        }
        if (__ldcg(&C->nnext[round & 1]) == 0) break;
        if (round >= M.maxRounds) {
            if (blockIdx.x == 0 && tid == 0) atomicCAS(&C->status, CT_OK, CT_ERR_TIMEOUT);
            break;
        }
    }

    // publish (every CTA left the loop at the same point): the per-table
    // results and resets by CTA 0 alone for a small network, by the whole grid
    // for a large one (then a barrier); CTA 0 releases the status word last
    const bool wide = M.ntables >= kWidePublish;
    if (!wide && blockIdx.x != 0) return;
    phase(6);
    __threadfence();
    __syncthreads();
    const int ptid = wide ? blockIdx.x * kThreads + tid : tid;
    const int pth = wide ? gridDim.x * kThreads : kThreads;
    int32_t* H = M.statusBlk;
    for (int t = ptid; t < M.ntables; t += pth) {
        Ctrl* Tc = M.tabs[t].ctrl;
        H[kModelHdr + 2 * t] = __ldcg(&Tc->trail_top);
        H[kModelHdr + 2 * t + 1] = __ldcg(&Tc->live_state);
        // leave every table's per-call counters clear
        Tc->live = 0u; Tc->live_in = 0u; Tc->words_in = 0u; Tc->nhard = 0u; Tc->nrows = 0; Tc->nscan = 0;
        Tc->hits = 0; Tc->local_found = 0; Tc->misses = 0; Tc->windows = 0; Tc->trail_added = 0;
        Tc->status = CT_OK;
    }
    uint32_t* outDom = reinterpret_cast<uint32_t*>(H + kModelHdr + 2 * M.ntables);
    for (int q = ptid; q < M.DWg; q += pth) outDom[q] = __ldcg(&M.dom[q]);
    const int nnodes = M.ntables / M.nodeTables;
    int32_t* outNode = H + kModelHdr + 2 * M.ntables + M.DWg;
    for (int q = ptid; q < nnodes; q += pth) {
        outNode[q] = __ldcg(&M.nodeStatus[q]);
        M.nodeStatus[q] = CT_OK;
    }
    int32_t* outSnap = outNode + nnodes;
    for (int t = ptid; t < M.ntables; t += pth) {
        outSnap[t] = __ldcg(&M.snapTaken[t]);
        M.snapTaken[t] = 0;
    }
    for (int v = ptid; v < 2 * M.nvars; v += pth) M.prunedBy[v] = -1;
    if (wide) {
        // every CTA's writes to the host-mapped block are visible system-wide
        // before CTA 0 publishes the status word
        __threadfence_system();
        if (!sync()) return;
        if (blockIdx.x != 0) return;
    }
    __syncthreads();
    if (tid == 0) {
        const int st = __ldcg(&C->status);
        H[1] = __ldcg(&C->rounds);
        H[2] = __ldcg(&C->props);
        H[3] = (int32_t)__ldcg(&C->hits);
        H[4] = (int32_t)__ldcg(&C->local);
        H[5] = (int32_t)__ldcg(&C->hard);
        H[6] = (int32_t)__ldcg(&C->windows);
        // filterDomains bytes as for one table: one word per residue hit, 128
        // words per window probed, 16 bytes per live chunk of every full scan
        const unsigned long long bf = __ldcg(&C->bytesFilter) + 4ull * __ldcg(&C->hits) +
                                      512ull * __ldcg(&C->windows);
        const unsigned long long bu = __ldcg(&C->bytesUpdate);
        H[8] = (int32_t)(bu & 0xffffffffull);
        H[9] = (int32_t)(bu >> 32);
        H[10] = (int32_t)(bf & 0xffffffffull);
        H[11] = (int32_t)(bf >> 32);
        C->hits = C->local = C->hard = C->windows = 0u;
        C->bytesUpdate = 0ull;
        C->bytesFilter = 0ull;
        C->nmiss[0] = C->nmiss[1] = 0;
        C->nscanAll[0] = C->nscanAll[1] = 0;
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
    for (int q = tid; q < S.arity; q += nth) D.other[q] = 0ull;
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

}  // namespace

// Launches of many tables (the batched searches' copies of a network) run 4
// CTAs per SM with 8 row loads in flight: a round's units are many and short,
// and twice the warps keep twice the loads in flight (batched search 1.2-1.3x
// nodes/s); smaller networks keep 2 CTAs per SM with 16 loads (4 CTAs per SM
// measured 6-7% slower there).
constexpr int kManyTables = 1024;

int max_coresident_model_blocks(int ntables) {
    int dev = 0, sms = 0, per = 0;
    const void* k = ntables >= kManyTables ? (const void*)ct_model_kernel<8, false, 4> : (const void*)ct_model_kernel<16, false>;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per * sms;
}

cudaError_t launch_model(const ModelDev& M, int grid, cudaStream_t s) {
    ModelDev m = M;
    void* args[] = {&m};
    const void* k = M.ntables >= kManyTables ? (const void*)ct_model_kernel<8, false, 4> : (const void*)ct_model_kernel<16, false>;
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, 0, s);
}

// Search mode: 4 CTAs per SM with 8 row loads in flight (twice the warps of
// the fixpoint launch: a round's units are many and short).
int max_coresident_search_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ct_model_kernel<8, true, 4>, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per * sms;
}

cudaError_t launch_model_search(const ModelDev& M, int grid, cudaStream_t s) {
    ModelDev m = M;
    void* args[] = {&m};
    return cudaLaunchCooperativeKernel((const void*)ct_model_kernel<8, true, 4>, dim3(grid), dim3(kThreads), args, 0, s);
}

// Level 0 of every slot (one CTA per slot): the root domains, and for every
// table an empty trail of trailFactor * W4 + 1024 entries in its own control
// block (the live count taken from the state copy's), mark 0 and the
// non-zero index as the state copy left it.
__global__ void ct_search_init_kernel(const __grid_constant__ ModelDev M, const TableDev* __restrict__ hostTabs,
                                      const SearchDev* __restrict__ Sp, const uint32_t* __restrict__ rootDom,
                                      int trailFactor) {
    const SearchDev& S = *Sp;
    const int s = blockIdx.x;
    const int tid = threadIdx.x;
    for (int q = tid; q < S.DWs; q += blockDim.x) S.levelDom[lvl(S, s, 0) * S.DWs + q] = rootDom[q];
    for (int k = tid; k < S.T; k += blockDim.x) {
        const int j = s * S.T + k;
        const TableDev& T = M.tabs[j];
        const int live = hostTabs[j].ctrl->live_state;
        int32_t* c = reinterpret_cast<int32_t*>(T.ctrl);
        for (int q = 0; q < (int)(sizeof(Ctrl) / sizeof(int32_t)); ++q) c[q] = 0;
        T.ctrl->cur_mark = -1;
        T.ctrl->trail_cap = trailFactor * T.W4 + 1024;
        T.ctrl->live_state = live;
        S.markAt[lvl(S, s, 0) * S.T + k] = 0;
        S.liveAt[lvl(S, s, 0) * S.T + k] = live;
        S.calls[j] = ModelTabCall{0, 0, 0, 0};
        uint32_t* snap = S.snapSeg + lvl(S, s, 0) * S.segTotal + S.segOff[k];
        for (int q = 0; q < T.nseg; ++q) snap[q] = T.segMask[q];
    }
    if (tid == 0) {
        S.depth[s] = 0;
        S.active[s] = 0;
        S.busy[s] = 0;
        S.firstOpen[s] = 0x7fffffff;
        M.nodeStatus[s] = CT_OK;
    }
}

cudaError_t launch_search_init(const ModelDev& M, const TableDev* hostTabs, const SearchDev& S,
                               const uint32_t* rootDom, int trailFactor, cudaStream_t s) {
    ct_search_init_kernel<<<S.B, 128, 0, s>>>(M, hostTabs, M.search, rootDom, trailFactor);
    return cudaGetLastError();
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

}  // namespace ctk
