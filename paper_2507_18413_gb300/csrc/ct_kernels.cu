// ct_kernels.cu -- CUDA kernels of Compact-Table propagation for sm_103a.
//
// One propagation (Algorithm 1, enforceGAC) is ONE cooperative launch whose
// CTAs step through these phases:
//   plan     Delta_x = lastDom_x & ~dom_x, s_val, s_sup, the delta/reset
//            choice of Algorithm 2 (delta iff |Delta| < |dom|) and the list
//            of supports rows to OR (row codes). For tables whose plan fits in
//            shared memory every CTA computes it for itself; otherwise CTA 0
//            writes it to global memory and a grid barrier follows.
//   update   Algorithm 2 on every live 128-bit chunk, over (segment, slice)
//            units: a segment is 32 chunks (lane l owns chunk 32s + l) and its
//            row list is cut into G = 1, 2, 4 or 8 slices held by adjacent
//            warps of one CTA, so that long lists spread over the whole grid;
//            each slice is walked in batches of 16 (or 8) independent 128-bit
//            loads per lane that bypass L1, a variable's OR is complemented on
//            the delta path and AND-ed in, and the slices of a segment are
//            combined in shared memory. Changed chunks go to the trail; the
//            segment's live mask (the non-zero index) is rebuilt with one warp
//            ballot.
//   -- grid barrier --
//   probe    Algorithm 1 line 5 (fail when currTable = 0), then one warp per
//            value of s_sup (Algorithm 3 with residues): the residue chunk
//            first (loaded beside the failure test); on a miss, up to four
//            32-chunk windows after it; values still unresolved go to the
//            hard list.
//   -- grid barrier --
//   publish  with no hard value, the CTA that arrived last at the barrier
//            writes lastDom's removals, the status block (mapped host memory)
//            and resets the per-call counters; otherwise every warp holds a
//            segment's live chunks and tests every hard value against them,
//            and the last CTA to finish removes the values no chunk supports,
//            stores new residues and publishes.
// Calls of at most U supports rows (positive local-plan tables with
// residues, at least half the chunks live at entry; ct_options.no_early_filter
// switches this off) run the probes
// beside the update instead: the update takes one round of the grid's warps
// (one segment per warp), the warps after it start on the values at once, and
// every chunk a probe tests is recomputed from its stored value and the
// call's rows (chunk_after: the stored value may be old or new, the result is
// the new one). One grid barrier then ends both phases and decides the
// failure from the update's live count; a value the windows left undecided
// waits (bounded) for the whole update and is searched again over the index
// it left when currTable has become sparse; the finalizing CTA writes lastDom
// (no CTA may write it before every plan is done).
// Grid barriers spin with a bounded iteration count; running out sets
// CT_ERR_TIMEOUT in the control block and every CTA returns.
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ct_device.cuh"

namespace ctk {


namespace {

// ---------------------------------------------------------------------------
// one CTA: apply Algorithm 3's removals, publish, reset the call counters
// ---------------------------------------------------------------------------

// Word of the control block read into each status header slot (-1: none),
// and the word subtracted from it (-1: none; the stamps are sent as ns since
// the start stamp, from their low words, and the start stamp as its low word).
#define CT_CW(f) (int16_t)(offsetof(Ctrl, f) / sizeof(int32_t))
#define CT_TLO(k) (int16_t)(offsetof(Ctrl, t) / sizeof(int32_t) + 2 * (k))
__constant__ int16_t kHdrWord[kStatusHdr] = {
    CT_CW(status), CT_CW(live), CT_CW(words_in), CT_CW(trail_top), CT_CW(misses), -1, CT_CW(hits), CT_CW(nrows),
    CT_CW(nval), CT_CW(nsup), CT_CW(ndelta), CT_CW(nreset), CT_CW(trail_added), CT_CW(live_in), CT_CW(local_found),
    CT_CW(nhard), CT_CW(windows), CT_TLO(1), CT_TLO(2), CT_TLO(3), CT_TLO(0), CT_CW(nscan), -1, -1};
__constant__ int16_t kHdrSub[kStatusHdr] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                                            CT_TLO(0), CT_TLO(0), CT_TLO(0), -1, -1, -1, -1};
#undef CT_CW
#undef CT_TLO
static_assert(kSlotStatus == 0 && kSlotLiveOut == 1 && kSlotWordsIn == 2 && kSlotTrailTop == 3 && kSlotMisses == 4 &&
                  kSlotPruned == 5 && kSlotHits == 6 && kSlotRowsOred == 7 && kSlotNval == 8 && kSlotNsup == 9 &&
                  kSlotNdelta == 10 && kSlotNreset == 11 && kSlotTrailAdded == 12 && kSlotLiveIn == 13 &&
                  kSlotLocal == 14 && kSlotHard == 15 && kSlotWindows == 16 && kSlotT1 == 17 && kSlotT2 == 18 &&
                  kSlotT3 == 19 && kSlotT4 == 20 && kSlotScan == 21 && kStatusHdr == 24,
              "status header slots as the tables above list them");

// Run by exactly one CTA once every other CTA is done with the call (the last
// to arrive at the final barrier, or the last to finish the full scan). Every
// counter of the call is read in one round of loads (thread k reads header
// slot k); t3 is the caller's stamp of the end of the probes (0: read it from
// the control block).
// nh < 0: the hard-value counts are read with the header, and with values
// left undecided for the full scan the CTA returns false without publishing
// (the hard values known unsupported are removed here).
// Nothing but this CTA writes the domains during a call, so the first hard
// entries (read whether or not they belong to this call, kept only below the
// count) and the domain words are loaded in the same round as the header;
// the removals go to a shared copy of the domains, which is what the host
// receives. localDom: sm.dom already holds the call's domains (local plan).
// lastDomHere: the filter ran beside the update, so no CTA wrote lastDom
// after the plans (a CTA may still be reading it in its plan before the
// barrier): this CTA writes it, the call's domains less the values it removes.
__device__ bool finalize(const TableDev& T, const VarLayout& V, uint32_t* __restrict__ dom, Smem& sm, int nh,
                         uint64_t t3, bool localDom, bool lastDomHere = false) {
    Ctrl* C = T.ctrl;
    const int tid = threadIdx.x;
    int32_t* H = T.statusBlk;
    __syncthreads();  // counters thread 0 of this CTA may have written just before
    const bool smemDom = localDom || T.DW <= kLocalMaxDW;
    int preRow = 0, preFc = 0;
    if (nh != 0) {
        if (tid < T.R) {
            preRow = __ldcg(&T.hardRow[tid]);
            preFc = __ldcg(&T.foundChunk[tid]);
        }
        if (!localDom && smemDom)
            for (int i = tid; i < T.arity; i += kThreads)
                for (int k = 0; k < V.nw(i); ++k) sm.dom[V.ld(i) + k] = __ldcg(&dom[V.off(i) + k]);
    }
    if (tid < kStatusHdr) {
        // one predicated load (two for a stamp difference) per slot, no
        // divergent branches: the header is read in one round
        const int32_t* cw = reinterpret_cast<const int32_t*>(C);
        const int a = kHdrWord[tid], b = kHdrSub[tid];
        int32_t v = a >= 0 ? __ldcg(cw + a) : 0;
        const int32_t w = b >= 0 ? __ldcg(cw + b) : 0;
        if (tid == kSlotHard && nh >= 0) v = nh;
        if (tid == kSlotT3 && t3) v = (int32_t)(uint32_t)t3;
        if (tid == kSlotEarly) v = lastDomHere ? 1 : 0;
        sm.scan[tid] = v - w;
    }
    if (tid == 0) sm.cnt[kCntPruned] = 0u;
    // bit i of sm.scan[kChgBase + i / 32]: scope variable i lost a value
    constexpr int kChgBase = 32;
    for (int q = tid; q < T.nChangedWords; q += kThreads) sm.scan[kChgBase + q] = 0;
    __syncthreads();
    CT_STAMP(15);
    int st = sm.scan[kSlotStatus];
    // With the filter beside the update, the failure (Algorithm 1 line 5) is
    // decided here from the update's live count, read in the header round.
    if (lastDomHere && st == CT_OK && sm.scan[kSlotLiveOut] == 0) st = CT_INFEASIBLE;
    if (nh < 0 && st == CT_OK && sm.scan[kSlotScan] > 0) return false;
    nh = sm.scan[kSlotHard];
    if (st == CT_OK && nh > 0) {
        uint32_t pruned = 0;
        for (int m = tid; m < nh; m += kThreads) {
            const int r = m == tid ? preRow : __ldcg(&T.hardRow[m]);
            const int fc = m == tid ? preFc : __ldcg(&T.foundChunk[m]);
            // positive tables: a chunk holding a support, or kNoChunk / kNoSupport;
            // negative tables: fc counts the valid forbidden tuples with the value
            const bool keep = T.negative ? (unsigned long long)fc < sm.other[T.rowVar[r]] : (fc >= 0 && fc != kNoChunk);
            if (keep) {
                if (!T.negative) T.residue[r] = fc;
            } else {
                // Algorithm 3 line 4: no live tuple carries the value.
                const int i = T.rowVar[r];
                const int a = r - V.row0(i);
                if (dom) atomicAnd(&dom[V.off(i) + (a >> 5)], ~(1u << (a & 31)));
                if (smemDom) atomicAnd(&sm.dom[V.ld(i) + (a >> 5)], ~(1u << (a & 31)));
                // a positive table's removed value carries no valid tuple, so
                // lastDom may drop it now; a negative table's value still has
                // valid forbidden tuples, which the next call removes as Delta;
                // a shard's value may be supported by another shard
                if (!T.negative && !T.shard && !lastDomHere)
                    atomicAnd(&T.lastDom[V.ld(i) + (a >> 5)], ~(1u << (a & 31)));
                atomicOr(reinterpret_cast<unsigned*>(&sm.scan[kChgBase + (i >> 5)]), 1u << (i & 31));
                ++pruned;
            }
        }
        if (pruned) atomicAdd(&sm.cnt[kCntPruned], pruned);
        __syncthreads();
        if (sm.cnt[kCntPruned]) {
            // The changed mask and the domains of the variables that lost values
            // go to the host (one thread per variable, all read at once).
            uint32_t* outDom = reinterpret_cast<uint32_t*>(H + kStatusHdr + T.nChangedWords);
            for (int q = tid; q < T.nChangedWords; q += kThreads) H[kStatusHdr + q] = sm.scan[kChgBase + q];
            for (int i = tid; i < T.arity; i += kThreads) {
                if (!((sm.scan[kChgBase + (i >> 5)] >> (i & 31)) & 1)) continue;
                for (int k = 0; k < V.nw(i); ++k)
                    outDom[V.ld(i) + k] = smemDom ? sm.dom[V.ld(i) + k] : __ldcg(&dom[V.off(i) + k]);
            }
        }
    }
    if (lastDomHere && st == CT_OK)
        for (int q = tid; q < T.DW; q += kThreads) T.lastDom[q] = sm.dom[q];
    // Header: one slot per thread.
    if (tid < kStatusHdr && tid != kSlotStatus) {
        int32_t v = sm.scan[tid];
        if (tid == kSlotPruned) v = (int32_t)sm.cnt[kCntPruned];
        else if (tid == kSlotT4) v = (int32_t)((uint32_t)gtimer() - (uint32_t)v);
        H[tid] = v;
    }
    __syncthreads();
    // Reset the per-call counters for the next call (after every read above).
    if (tid == 0) {
        C->live = 0u; C->live_in = 0u; C->words_in = 0u; C->nhard = 0u; C->done = 0u; C->nscan = 0; C->tuples = 0u;
        C->upd_done = 0u;
        C->hits = 0; C->trail_added = 0; C->local_found = 0; C->misses = 0; C->windows = 0;
        C->nval = 0; C->ndelta = 0; C->nreset = 0; C->nsup = 0; C->nrows = 0;
        C->status = CT_OK;
        // Everything written above reaches the host before the word that publishes it.
        st_release_sys(&H[kSlotStatus], st);
    }
    return true;
}

// The residue test of value r with its residue chunk already loaded (lane 0),
// then Algorithm 3's window search on a miss: over the chunks that follow the
// residue while most chunks are live, over the LIVE chunks that follow it
// (found through the non-zero index) when fewer than half are, where a value
// whose windows covered every live chunk is known unsupported without a scan.
__device__ __forceinline__ void probe_loaded(const TableDev& T, int r, bool present, int res, const uint4& supRes,
                                             const uint4& curRes, bool sparse, uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31;
    if (!present) return;
    if (T.useResidues) {
        const bool hit = __shfl_sync(0xffffffffu, lane == 0 && nz(and4(supRes, curRes)), 0);
        if (hit) {
            if (lane == 0) atomicAdd(&s_cnt[kCntHits], 1u);
            return;
        }
    }
    if (sparse) probe_miss<true, kModelProbes>(T, r, res, s_cnt);
    else probe_miss<false, kLocalProbes>(T, r, res, s_cnt);
}

// A value of s_sup probed beside the update (r and res uniform over the
// warp): its residue chunk and, on a miss, the windows after it, every chunk
// recomputed from the call's row codes (chunk_after, E >= nrows rows). The
// sparse/dense choice of windows is the state's at entry; when they leave the
// value undecided and the update has made currTable sparse (the live count is
// final once every CTA has released its update), the value is searched again
// over the live chunks of the index the update left, after waiting for it.
template <int E>
__device__ __forceinline__ void probe_early(const TableDev& T, int r, bool present, int res, const int32_t* codes,
                                            int nrows, bool sparse, unsigned limit, uint32_t* s_cnt) {
    const int lane = threadIdx.x & 31;
    if (!present) return;
    bool hit = false;
    if (lane == 0) hit = nz(and4(ld_sup(T.sup + (size_t)r * T.W4 + res), chunk_after<E>(T, codes, nrows, res)));
    if (__shfl_sync(0xffffffffu, hit, 0)) {
        if (lane == 0) atomicAdd(&s_cnt[kCntHits], 1u);
        return;
    }
    int o = sparse ? probe_windows<true, kModelProbes, E>(T, r, res, s_cnt, codes, nrows)
                   : probe_windows<false, kLocalProbes, E>(T, r, res, s_cnt, codes, nrows);
    if (o == kProbeUndecided && wait_update_done(T.ctrl, limit) && 2u * __ldcg(&T.ctrl->live) < (uint32_t)T.W4)
        o = probe_windows<true, kModelProbes>(T, r, res, s_cnt);
    note_probe(T, r, o, s_cnt);
}

// Per-CTA counters of a phase into the control block (zero counts skipped).
__device__ __forceinline__ void flush_update_counters(Ctrl* C, Smem& sm) {
    if (sm.cnt[kCntLive]) atomicAdd(&C->live, sm.cnt[kCntLive]);
    if (sm.cnt[kCntLiveIn]) atomicAdd(&C->live_in, sm.cnt[kCntLiveIn]);
    if (sm.cnt[kCntWords]) atomicAdd(&C->words_in, sm.cnt[kCntWords]);
    if (sm.cnt[kCntTrail]) atomicAdd(&C->trail_added, (int)sm.cnt[kCntTrail]);
    if (sm.cnt[kCntTuples]) atomicAdd(&C->tuples, sm.cnt[kCntTuples]);
}

// ---------------------------------------------------------------------------
// the propagation kernel
// ---------------------------------------------------------------------------
template <bool kLocal, int U, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
ct_propagate_kernel(const __grid_constant__ TableDev T, uint32_t* __restrict__ dom,
                    const int32_t* __restrict__ domOff, const __grid_constant__ CallParams P) {
    __shared__ Smem sm;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    SliceSmem& parts = *reinterpret_cast<SliceSmem*>(s_dyn);
    Ctrl* C = T.ctrl;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    const VarLayout V(T, P.domOff, domOff);
    // Host-buffer calls of local-plan tables pass the domains as parameters:
    // the plan reads them there, and the result leaves through the status
    // block alone (the finalizing CTA publishes it from its shared copy).
    const bool domParams = kLocal && P.domInParams;
    const uint32_t* domIn = domParams ? P.domWords : dom;
    uint32_t* domOut = domParams ? nullptr : dom;
    GridBarrier bar;
    bar_init(bar, &C->bar_count, &C->bar_base, &C->status, P.spinLimit ? P.spinLimit : kBarrierSpinLimit);
    if (blockIdx.x == 0 && tid == 0) C->t[0] = gtimer();
    CT_STAMP(0);

    // Prologue loads that do not depend on the plan: the first segment of the
    // warp when every warp takes a whole segment, and the residue (with its
    // supports chunk) of the first value it probes.
    SegState seg0;
    if (gwarp < T.nseg) seg0 = load_segment(T, gwarp, P.mark);
    // (the supports chunk at the residue is loaded after the plan, so that the
    // warp does not wait for the residue before the plan's loads)
    int res0 = 0;
    uint4 supRes0 = make_uint4(0u, 0u, 0u, 0u);
    if (T.useResidues && gwarp < T.R && lane == 0) res0 = T.residue[gwarp];
    // With the filter beside the update (a call of at most U rows: one warp
    // per segment, one round), the warps after the round's segments take the
    // values first: warp g starts at value (g - nseg) mod nwarps.
    const int pfirstE = (gwarp - T.nseg % nwarps + nwarps) % nwarps;
    int resE = 0;
    if (kLocal && P.early > 0 && T.useResidues && pfirstE < T.R && lane == 0) resE = T.residue[pfirstE];

    CT_STAMP(19);
    // plan (CTA 0 also snapshots lastDom into the levels saved since the last call)
    int nrows;
    bool ok;
    if (kLocal) {
        const bool snap = blockIdx.x == 0;
        plan(T, V, domIn, sm.k, sm.rowOff, sm.sup, sm.codes, sm.dom, sm, snap ? P.snapFrom : 0, snap ? P.snapTo : 0);
        ok = !(sm.flags[0] || sm.flags[1]);
        nrows = sm.flags[6];
        if (T.negative && ok) {
            // every value of x_i is excluded when all prod_{j != i} |D_j| combinations
            // with it are forbidden: the products, saturated at 2^62
            if (tid == 0) {
                const unsigned long long cap = 1ull << 62;
                auto mul = [&](unsigned long long a, unsigned long long b) {
                    return (b != 0 && a > cap / b) ? cap : a * b;
                };
                unsigned long long pre = 1ull;
                for (int i = 0; i < T.arity; ++i) {
                    sm.other[i] = pre;
                    pre = mul(pre, (unsigned long long)sm.nd[i]);
                }
                unsigned long long suf = 1ull;
                for (int i = T.arity - 1; i >= 0; --i) {
                    sm.other[i] = mul(sm.other[i], suf);
                    suf = mul(suf, (unsigned long long)sm.nd[i]);
                }
            }
            __syncthreads();
        }
        if (blockIdx.x == 0 && tid == 0) {
            C->nval = sm.flags[2]; C->ndelta = sm.flags[3]; C->nreset = sm.flags[4]; C->nsup = sm.flags[5];
            C->nrows = nrows;
            if (!ok) C->status = sm.flags[0] ? CT_ERR_STATE : CT_INFEASIBLE;
        }
    } else {
        if (blockIdx.x == 0) {
            plan(T, V, dom, T.planK, T.planRowOff, T.varSup, T.codes, nullptr, sm, P.snapFrom, P.snapTo);
            if (tid == 0) {
                C->nval = sm.flags[2]; C->ndelta = sm.flags[3]; C->nreset = sm.flags[4]; C->nsup = sm.flags[5];
                C->nrows = sm.flags[6];
                if (sm.flags[0] || sm.flags[1]) C->status = sm.flags[0] ? CT_ERR_STATE : CT_INFEASIBLE;
            }
        }
        if (!bar_sync(bar, &sm.flag[0])) return;
        ok = __ldcg(&C->status) == CT_OK;
        nrows = __ldcg(&C->nrows);
        const int staged = min(nrows, kCodeCap);
        for (int q = tid; q < staged; q += kThreads) sm.codes[q] = __ldcg(&T.codes[q]);
    }
    if (blockIdx.x == 0 && tid == 0) C->t[1] = gtimer();
    CT_STAMP(1);
    // Filter beside the update (Algorithm 3 on the chunks Algorithm 2 leaves,
    // each recomputed from the call's rows: chunk_after): for calls of at most
    // U rows on positive local-plan tables with residues, while at least half
    // the chunks are live at entry (in a sparse state the probes beside the
    // update would walk the index before the update, whose dying chunks cost
    // windows: measured slower there). The probes need no
    // barrier after the update; the one barrier after them also decides the
    // failure (Algorithm 1 line 5) from the update's live count. Every CTA
    // takes the same decision (each computed the same plan).
    const bool early = kLocal && ok && nrows > 0 && nrows <= U && nrows <= P.early && !T.negative && !T.shard &&
                       T.useResidues && 2 * P.prevLive >= T.W4;
    if (T.useResidues && gwarp < T.R && lane == 0 && !early)
        supRes0 = ld_sup(T.sup + (size_t)gwarp * T.W4 + res0);

    uint4 curRes0 = make_uint4(0u, 0u, 0u, 0u);
    bool sparse = 2 * P.prevLive < T.W4;  // fewer than half the chunks live (after the update: recomputed)
    if (!ok || (nrows == 0 && !T.negative)) {
        // Nothing to update: currTable stays as it is. Pending level snapshots
        // of the index are still taken.
        for (int seg = gwarp; seg < T.nseg; seg += nwarps) {
            const uint32_t mk = seg == gwarp ? seg0.mask : T.segMask[seg];
            for (int l = P.snapFrom + lane; l < P.snapTo; l += 32) T.levelSeg[(size_t)l * T.nseg + seg] = mk;
        }
        if (!ok) {
            // Domain error or empty domain: publish without filtering.
            if (blockIdx.x == 0) finalize(T, V, domOut, sm, 0, 0ull, kLocal);
            return;
        }
        if (blockIdx.x == 0 && tid == 0) {
            C->live = (uint32_t)P.prevLive;
            C->live_in = (uint32_t)P.prevLive;
            C->t[2] = C->t[1];
        }
        if (T.useResidues && gwarp < T.R && lane == 0) curRes0 = __ldcg(T.curr + res0);
    } else {
        // update (Algorithm 2): the row list of a segment is cut into G slices,
        // G a power of two and at most P.maxSplit, as large as keeps every
        // (segment, slice) unit in one round of the grid's warps and no larger
        // than one batch of U rows per slice needs; warp w of a round takes
        // slice w % G of segment (round base + w) / G, and the slices of one
        // segment, held by the G adjacent warps of one CTA, are combined in
        // shared memory.
        if (tid < 12) sm.cnt[tid] = 0u;
        int G = 1, lg = 0;
        {
            const int need = (nrows + U - 1) / U;
            while (G < P.maxSplit && G < need && (T.nseg << (lg + 1)) <= nwarps) {
                G <<= 1;
                ++lg;
            }
        }
        const int units = T.nseg << lg;
        const int per = (nrows + G - 1) >> lg;  // rows per slice
        __syncthreads();
        CT_STAMP(20);
        const int cap = __ldcg(&C->trail_cap);
        // Rounds of one unit per warp; every warp of a CTA runs every round so
        // that the trail reservation and the slice combination can
        // synchronise the CTA.
        for (int base = blockIdx.x * kWarps; base < units; base += nwarps) {
            const int u = base + warp;
            const int seg = u >> lg, slice = u & (G - 1);
            TrailItem it;
            it.need = false;
            SegState S;
            S.mask = 0u;
            TrailSlots slots;
            slots.cand = 0u;
            if (u < units) {
                S = (G == 1 && seg == gwarp) ? seg0 : load_segment(T, seg, P.mark);
                if (slice == 0) {
                    // levels saved since the last call snapshot the index as it is now
                    for (int l = P.snapFrom + lane; l < P.snapTo; l += 32) T.levelSeg[(size_t)l * T.nseg + seg] = S.mask;
                    slots.cand = __ballot_sync(0xffffffffu, P.mark >= 0 && ((S.mask >> lane) & 1u) && S.lp < P.mark);
                }
            }
            if (lane == 0) sm.trw[warp] = __popc(slots.cand);
            CT_STAMP(21);
            __syncthreads();
            int ctaBase = 0;  // thread 0: the CTA's block of slots, waited for after the row loads
            if (tid == 0) {
                int tot = 0;
                for (int k = 0; k < kWarps; ++k) {
                    const int c = sm.trw[k];
                    sm.trw[k] = tot;
                    tot += c;
                }
                if (tot) ctaBase = atomicAdd(&C->trail_top, tot);
            }
            CT_STAMP(8);
            uint4 acc = make_uint4(~0u, ~0u, ~0u, ~0u);
            if (G == 1) {
                if (S.mask != 0u)
                    acc = slice_rows<U, false, false>(T, seg, (S.mask >> lane) & 1u, S.cur, 0, nrows, sm.codes,
                                                      nullptr, 0);
            } else {
                if (S.mask != 0u) {
                    const int qa = min(nrows, slice * per);
                    slice_rows<U, false, true>(T, seg, (S.mask >> lane) & 1u, S.cur, qa, min(nrows, qa + per),
                                               sm.codes, &parts, warp);
                }
                __syncthreads();
                if (S.mask != 0u && slice == 0) acc = combine_slices(parts, warp, G);
            }
            CT_STAMP(9);
            if (tid == 0) sm.trBase = ctaBase;
            __syncthreads();
            CT_STAMP(10);
            if (S.mask != 0u && slice == 0) {
                finish_segment(T, P.mark, seg, S, acc, sm.cnt, &sm.cnt[kCntTuples], it);
                slots.base = sm.trBase + sm.trw[warp];
                trail_write(T, slots, it, cap, sm.cnt);
            }
            __syncthreads();  // the slot counts and the parts are rewritten by the next round
        }
        __syncthreads();
        CT_STAMP(2);
        if (tid == 0) flush_update_counters(C, sm);
        if (early) {
            __syncthreads();  // the counters are read before the probes clear them
            // this CTA's part of the update and its counts, released to the
            // probes that wait for the whole update (wait_update_done)
            if (tid == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&C->upd_done) : "memory");
        }
    }
    if (ok && (nrows > 0 || T.negative) && !early) {
        const int r1 = bar_sync(bar, &sm.flag[0]);
        if (!r1) return;
        CT_STAMP(3);
        if (r1 == 2 && tid == 0) C->t[2] = gtimer();
        // Algorithm 1 line 5: fail when currTable is all zero (a negative
        // table with no valid forbidden tuple forbids nothing; an empty shard
        // supports no value, which the filter finds). The residue chunk of the
        // warp's first probe is loaded beside the failure test.
        if (T.useResidues && gwarp < T.R && lane == 0) curRes0 = __ldcg(T.curr + res0);
        const int st1 = __ldcg(&C->status);
        const uint32_t live1 = __ldcg(&C->live);
        sparse = 2u * live1 < (uint32_t)T.W4;
        if (st1 != CT_OK || (!T.negative && !T.shard && live1 == 0u)) {
            if (r1 == 2) {
                if (tid == 0 && st1 == CT_OK) C->status = CT_INFEASIBLE;
                __syncthreads();
                finalize(T, V, domOut, sm, 0, 0ull, kLocal);
            }
            return;
        }
    }

    // residue probes (Algorithm 3)
    if (tid < 12) sm.cnt[tid] = 0u;
    __syncthreads();
    // lastDom := the domains of this call (values pruned below are cleared
    // again by the finalizing CTA).
    if (blockIdx.x == 0 && !early) {
        if (kLocal) {
            for (int q = tid; q < T.DW; q += kThreads) T.lastDom[q] = sm.dom[q];
        } else {
            for (int i = tid; i < T.arity; i += kThreads)
                for (int q = 0; q < V.nw(i); ++q) T.lastDom[V.ld(i) + q] = dom[V.off(i) + q];
        }
    }
    if (kLocal && T.negative) {
        // Negative tables: a value loses its support only when the valid
        // forbidden tuples carrying it are all prod_{j != i} |D_j| combinations;
        // values whose product exceeds the valid tuples keep it without a count.
        const unsigned long long liveT = __ldcg(&C->tuples);
        for (int r = blockIdx.x * kThreads + tid; r < T.R; r += gridDim.x * kThreads) {
            const int i = __ldg(&T.rowVar[r]);
            const int a = r - V.row0(i);
            const bool present = (sm.dom[V.ld(i) + (a >> 5)] >> (a & 31)) & 1u;
            if (present && sm.other[i] <= liveT) {
                const unsigned m = atomicAdd(&C->nhard, 1u);
                T.hardRow[m] = r;
                T.foundChunk[m] = 0;
                atomicAdd(&C->nscan, 1);
            }
        }
    } else if (early) {
        for (int r = pfirstE; r < T.R; r += nwarps) {
            const int i = __ldg(&T.rowVar[r]);
            const int a = r - V.row0(i);
            const bool present = sm.sup[i] && ((sm.dom[V.ld(i) + (a >> 5)] >> (a & 31)) & 1u);
            int res = resE;
            if (r != pfirstE && present && lane == 0) res = T.residue[r];
            res = __shfl_sync(0xffffffffu, res, 0);
            if (nrows <= 4) probe_early<4>(T, r, present, res, sm.codes, nrows, sparse, bar.limit, sm.cnt);
            else probe_early<U>(T, r, present, res, sm.codes, nrows, sparse, bar.limit, sm.cnt);
        }
    } else
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
        uint4 sr = supRes0, cr = curRes0;
        if (r != gwarp && T.useResidues && present && lane == 0) {
            res = T.residue[r];
            sr = ld_sup(T.sup + (size_t)r * T.W4 + res);
            cr = __ldcg(T.curr + res);
        }
        res = __shfl_sync(0xffffffffu, res, 0);
        probe_loaded(T, r, present, res, sr, cr, sparse, sm.cnt);
    }
    __syncthreads();
    if (tid == 0) {
        if (sm.cnt[kCntHits]) atomicAdd(&C->hits, (int)sm.cnt[kCntHits]);
        if (sm.cnt[kCntLocal]) atomicAdd(&C->local_found, (int)sm.cnt[kCntLocal]);
        if (sm.cnt[kCntMiss]) atomicAdd(&C->misses, (int)sm.cnt[kCntMiss]);
        if (sm.cnt[kCntWin]) atomicAdd(&C->windows, (int)sm.cnt[kCntWin]);
    }
    CT_STAMP(4);
    const int r2 = bar_sync(bar, &sm.flag[0]);
    if (!r2) return;
    CT_STAMP(5);
    const uint64_t t3 = r2 == 2 ? gtimer() : 0ull;
    if (early) {
        // Algorithm 1 line 5 after the update, whose counts every CTA flushed
        // before this barrier: the finalizing CTA decides it in its header
        // round (finalize), the others return on a failure (or once the
        // finalizing CTA has cleared the count, having needed no scan).
        if (r2 == 2 && tid == 0) C->t[2] = t3;
        if (r2 != 2 && (__ldcg(&C->status) != CT_OK || __ldcg(&C->live) == 0u)) return;
    }
    // The CTA that arrived last reads the hard-value counts with the counters
    // it publishes: with none left undecided (every value kept its support,
    // or its windows covered every live chunk) it removes the unsupported
    // values and publishes, and the others are done.
    if (r2 == 2 && finalize(T, V, domOut, sm, -1, t3, kLocal, early)) {
        CT_STAMP(6);
        return;
    }
    if (__ldcg(&C->nscan) == 0) return;
    const int nh = (int)__ldcg(&C->nhard);
    if (r2 == 2 && tid == 0) C->t[3] = t3;
    // full scan of the hard values
    CT_STAMP(11);
    {
        const int staged = min(nh, kCodeCap);
        for (int q = tid; q < staged; q += kThreads) sm.codes[q] = __ldcg(&T.hardRow[q]);
        __syncthreads();
        CT_STAMP(12);
        if (T.negative) {
            for (int seg = gwarp; seg < T.nseg; seg += nwarps) count_segment(T, seg, nh, sm.codes);
        } else {
            for (int seg = gwarp; seg < T.nseg; seg += nwarps) scan_segment<U>(T, seg, nh, sm.codes);
        }
    }
    // last-block-done
    CT_STAMP(13);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(&C->done, 1u);
        sm.flag[1] = (t == gridDim.x - 1);
    }
    __syncthreads();
    CT_STAMP(14);
    if (!sm.flag[1]) return;
    __threadfence();
    finalize(T, V, domOut, sm, nh, 0ull, kLocal, early);
    CT_STAMP(7);
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

// Static and dynamic shared memory together exceed 48 KB: opt in once per
// kernel variant before its first occupancy query or launch.
template <bool L, int U, int B>
cudaError_t allow_slice_smem() {
    static const cudaError_t e = cudaFuncSetAttribute((const void*)ct_propagate_kernel<L, U, B>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)sizeof(SliceSmem));
    return e;
}

template <bool L, int U, int B>
cudaError_t launch_coop(const TableDev& T, int grid, uint32_t* dom, const int32_t* domOff, const CallParams& P,
                        cudaStream_t s) {
    const cudaError_t e = allow_slice_smem<L, U, B>();
    if (e != cudaSuccess) return e;
    TableDev t = T;
    CallParams p = P;
    void* args[] = {&t, &dom, (void*)&domOff, &p};
    return cudaLaunchCooperativeKernel((const void*)ct_propagate_kernel<L, U, B>, dim3(grid), dim3(kThreads), args,
                                       sizeof(SliceSmem), s);
}

template <bool L, int U, int B>
int coresident() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (allow_slice_smem<L, U, B>() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ct_propagate_kernel<L, U, B>, kThreads,
                                                      sizeof(SliceSmem)) != cudaSuccess)
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

#ifdef CT_PHASE_TRACE
extern "C" int ct_trace_read(unsigned long long* out, int n) {
    if (n > kTraceCtas * kTraceStamps) n = kTraceCtas * kTraceStamps;
    return cudaMemcpyFromSymbol(out, g_ct_trace, (size_t)n * sizeof(unsigned long long)) == cudaSuccess ? 0 : -3;
}
#endif

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

// One streaming read of n16 chunks (ct_read_ceiling): U independent 128-bit
// loads per thread and round, grid-strided; the XOR of what was read decides
// a store that never happens in practice, so the loads are not dropped.
__device__ uint32_t g_ct_read_sink;
template <int U>
__global__ void __launch_bounds__(256) ct_read_kernel(const uint4* __restrict__ a, size_t n16) {
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    uint32_t x = 0u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += nth * U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_sup_pred(a + i + (size_t)u * nth, i + (size_t)u * nth < n16);
#pragma unroll
        for (int u = 0; u < U; ++u) x ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (x == 0x9e3779b9u) g_ct_read_sink = x;
}

cudaError_t launch_read_ceiling(const uint4* p, size_t n16, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    ct_read_kernel<8><<<4 * sms, 256, 0, s>>>(p, n16);
    return cudaGetLastError();
}

cudaError_t launch_copy_words(uint32_t* dst, const uint32_t* src, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    if (grid > 1024) grid = 1024;
    ct_copy_words_kernel<<<grid, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace ctk
