// ct_internal.cuh -- device layout of a Compact-Table constraint and the
// launchers of its kernels. Private to libct.so.
//
// Device layout of one table (all resident in HBM for the table's lifetime):
//   sup      uint4 [R][W4]   supports rows (Sec. 2, Table 1(b)), value-major:
//                             row jmp[i] + v - lo[i] holds bit j for every
//                             tuple j with tau_j[i] == v; 16-byte aligned rows
//   curr     uint4 [W4]      currTable (Sec. 2, Table 1(c)) as 128-bit chunks
//   segMask  uint32 [nseg]   non-zero index: bit l of segMask[s] is set iff
//                             chunk 32*s + l of currTable is non-zero
//   lastpos  int32 [W4]      trail position of the latest entry of each chunk
//   trailKey int2  [cap]     (chunk, previous trail position of that chunk)
//   trailOld uint4 [cap]     chunk value before the change
//   residue  int32 [R]       last chunk found supporting each row (a hint)
//   lastDom  uint32 [DW]     domains seen at the end of the last call
//                             (lastSizes of Algorithm 1, kept as bitsets)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ct.h"

namespace ctk {

constexpr int kMaxArity = 2048;
constexpr int kMaxDomSize = 65536;
constexpr int kThreads = 256;          // threads per CTA of the propagation kernel
constexpr int kWarps = kThreads / 32;
constexpr int kCodeCap = 4096;         // row codes staged in shared memory per CTA
constexpr int kLocalMaxArity = 512;    // every CTA plans for itself up to this arity,
constexpr int kLocalMaxDW = 2048;      // this many domain words and kCodeCap rows
constexpr int kStatusHdr = 24;         // int32 slots before the changed mask
constexpr int32_t kNoChunk = 0x7fffffff;
constexpr int32_t kNoSupport = -2;         // hard-list mark: no live chunk supports the value (no scan needed)
// Row code of the update plan: supports row | flags.
constexpr int32_t kCodeLast = 1 << 30;   // last row of its variable: apply the mask
constexpr int32_t kCodeDelta = 1 << 29;  // variable on the delta path: mask = ~OR(rows)
constexpr int32_t kCodeRow = (1 << 29) - 1;
constexpr int kLocalProbes = 4;          // windows of 32 chunks searched after a residue miss (one table)
constexpr int kModelProbes = 8;          // the same in the network kernel (live chunks)
constexpr int kWidePublish = 2048;       // network kernel: tables from which the whole grid publishes
constexpr int kWindowGroups = 8;         // index segments read for them: at most 8 x 32 (8,192 chunks)
constexpr unsigned kBarrierSpinLimit = 1u << 24;  // default polls of a grid-barrier wait
constexpr int kHostWaitMs = 2000;      // host poll of the status word before a stream sync
constexpr int kParamArity = 16;        // scopes up to this arity carry their layout in kernel parameters
constexpr int kWarpPlanWords = 4;      // domain words per variable a one-warp plan holds in registers
constexpr int kParamDomWords = 16;     // host-buffer calls of up to this many domain words pass them as parameters

// Status block header slots (written to mapped host memory after every call).
enum StatusSlot {
    kSlotStatus = 0,
    kSlotLiveOut = 1,
    kSlotWordsIn = 2,
    kSlotTrailTop = 3,
    kSlotMisses = 4,
    kSlotPruned = 5,
    kSlotHits = 6,
    kSlotRowsOred = 7,
    kSlotNval = 8,
    kSlotNsup = 9,
    kSlotNdelta = 10,
    kSlotNreset = 11,
    kSlotTrailAdded = 12,
    kSlotLiveIn = 13,
    kSlotLocal = 14,
    kSlotHard = 15,
    kSlotWindows = 16,
    kSlotT1 = 17,  // ns from kernel start to: plan done,
    kSlotT2 = 18,  // update done (after the barrier),
    kSlotT3 = 19,  // probes done (after the barrier),
    kSlotT4 = 20,  // finalize
    kSlotScan = 21,  // hard values left undecided by the windows (the full scan's)
    kSlotEarly = 22,  // 1: the filter ran beside the update (one grid barrier)
};

// Per-table control block: persistent state and per-call counters.
struct Ctrl {
    int32_t status;
    int32_t trail_top;   // persistent: entries in use
    int32_t cur_mark;    // persistent: trail_top at the newest save, -1 with no level
    int32_t trail_cap;
    uint32_t live;       // per call: chunks alive after updateTable
    uint32_t live_in;    // per call: chunks live at entry
    uint32_t words_in;   // per call: non-zero 32-bit words at entry
    uint32_t nhard;      // per call: values left for the full index scan
    uint32_t done;       // last-block-done ticket
    int32_t nrows;       // rows in the update plan
    int32_t nval, ndelta, nreset, nsup;
    int32_t hits, pruned, trail_added, local_found, misses, windows;
    int32_t live_state;  // live chunks after the last update (kept across calls)
    int32_t nscan;       // per call: hard values that need the full scan (the others are known unsupported)
    uint32_t tuples;     // per call, negative tables: valid tuples after the update
    uint32_t upd_done;   // per call: CTAs done with the update (a filter beside it may wait on it)
    uint64_t t[4];       // %globaltimer stamps of CTA 0 (diagnostics)
    // The barrier words on a line of their own: the arrivals and polls of
    // every CTA would otherwise hold up the finalizing CTA's reads of the
    // counters above.
    alignas(128) uint32_t bar_count;  // grid barrier arrivals (only grows)
    uint32_t bar_base;                // grid barrier count at the start of the next launch
};

// Everything a kernel needs, passed by value.
struct TableDev {
    const uint4* sup;        // [R][W4] supports rows (short tuples in every row of a wildcard position)
    const uint4* supDelta;   // rows OR-ed on the delta path: sup itself, or without the wildcards
    uint4* curr;
    uint32_t* segMask;
    int32_t* lastpos;
    int2* trailKey;
    uint4* trailOld;
    int32_t* residue;
    uint32_t* lastDom;
    Ctrl* ctrl;
    int32_t* codes;          // [R] update plan: row codes (global plan mode)
    int32_t* planK;          // [arity] rows to OR | delta flag (global plan mode)
    int32_t* planRowOff;     // [arity] first code of each variable (global plan mode)
    int32_t* varSup;         // [arity] 1 if |dom| > 1 (s_sup, global plan mode)
    unsigned long long* other;  // [arity] negative tables in the network kernel: product of the
                                // other scope domains' sizes (saturated), written by the plan
    int32_t* hardRow;        // [R] values left for the full scan
    int32_t* foundChunk;     // [R]
    const int32_t* rowVar;   // [R] scope position of each row
    const int32_t* varRow0;  // [arity+1] first row of each variable (_supportJmp)
    const int32_t* varNW;    // [arity] words of each domain
    const int32_t* varLD;    // [arity] offset of each domain in lastDom / packed layout
    int32_t* statusBlk;      // [kStatusHdr + nChangedWords + DW], mapped host memory
    uint32_t* levelSeg;      // [levelCap][nseg] live masks
    uint32_t* levelDom;      // [levelCap][DW]
    int32_t arity, R, W4, nseg, S, DW, nChangedWords, useResidues;
    int32_t negative;        // 1: the tuples are forbidden (negative table)
    int32_t shard;           // 1: a word-range shard (one-table kernel only): no failure on an
                             // empty currTable, lastDom keeps the call's input domains
    int32_t warpPlan;        // 1: the network kernel plans it with one warp (positive, arity
                             // <= 32, every domain <= kWarpPlanWords words)
    // Scopes of at most kParamArity variables: words, lastDom offset and first
    // supports row of each variable, so that the plan reads no global table.
    int32_t pNW[kParamArity], pLD[kParamArity], pRow0[kParamArity];
};

// Per-call parameters of the propagation kernel.
struct CallParams {
    int32_t mark;      // trail position of the newest saved level, -1 with no level
    int32_t snapFrom;  // levels [snapFrom, snapTo) were saved since the last call:
    int32_t snapTo;    // the kernel snapshots the index and lastDom into them first
    int32_t prevLive;  // live chunks of the current state (reported when no row is OR-ed)
    uint32_t spinLimit;  // polls of a grid-barrier wait before it gives up (CT_ERR_TIMEOUT)
    int32_t maxSplit;    // most warps that share one segment's row list (1, 2, 4 or 8)
    int32_t domOff[kParamArity];  // word offset of each scope domain (arity <= kParamArity)
    int32_t domInParams;          // 1: the domains are domWords (local plan only); the result
                                  // leaves through the status block alone
    uint32_t domWords[kParamDomWords];
    int32_t early;     // calls of at most min(early, U) rows filter beside the update (0: never; local plan)
};

// Dynamic shared memory of the propagation kernel: the partial results of the
// warps that share a segment's row list (updateTable split over warps).
struct SliceSmem {
    uint4 acc[kWarps][32];   // AND of the masks of the variables whose rows all lie in the slice
    uint4 head[kWarps][32];  // OR of the slice's rows of a variable that began before the slice
    uint4 tail[kWarps][32];  // OR of the slice's rows of a variable that goes on after the slice
    int32_t headKind[kWarps];   // 0 none; 1 that variable ends in the slice; 2 the slice lies inside it
    int32_t headDelta[kWarps];  // the head variable is on the delta path
    int32_t tailKind[kWarps];   // 1: an open tail
};
constexpr int kMaxSplit = kWarps;  // warps of one CTA that may share a segment

// ---------------------------------------------------------------------------
// A network of tables propagated to its fixpoint in one launch.
// ---------------------------------------------------------------------------
constexpr int kModelMaxTables = 1 << 20;
constexpr int kPrefixSmem = 2047;      // rounds of up to this many tables keep their prefix arrays in shared memory
constexpr int kModelHdr = 12;          // status block: header ints before the per-table pairs
// header: [0] status, [1] rounds, [2] table propagations, [3] residue hits,
// [4] window hits, [5] hard values, [6] windows, [8..9] updateTable bytes,
// [10..11] filterDomains bytes (64-bit, little end first)

struct RestoreDesc {
    int32_t table, level, mark, top;
};

struct ModelTabCall {
    int32_t mark;      // trail position of the table's newest level, -1 with none
    int32_t snapFrom;  // pending level snapshots [snapFrom, snapTo)
    int32_t snapTo;
    int32_t pad;
};

struct ModelCtrl {
    int32_t status;
    int32_t nwork;       // tables of the first round (when not passed in nworkIn)
    int32_t rounds;
    int32_t props;       // table propagations done
    int32_t nnext[2];    // tables of round r collected in nnext[r & 1] by round r - 1
    uint32_t hits;       // values whose residue still had a support
    uint32_t local;      // values found in the windows after the residue
    uint32_t hard;       // values left for the full index scan
    uint32_t windows;    // windows probed
    int32_t nmiss[2];    // residue misses queued in round r, in nmiss[r & 1]
    int32_t nscanAll[2]; // values of round r left for full scans, in nscanAll[r & 1]
    unsigned long long bytesUpdate;  // algorithmic bytes of updateTable: 4 * words at entry * (rows + 2)
    unsigned long long bytesFilter;  // of the full scans: 16 * hard values * live chunks
    // on a line of their own, away from the counters every CTA reads after a barrier
    alignas(128) uint32_t bar_count;  // grid barrier arrivals (only grows)
    uint32_t bar_base;                // grid barrier count at the start of the next launch
};

// ---------------------------------------------------------------------------
// The batched search run on the device (ct_search_batch_device): B slots, each
// a copy of the network (T tables, nv variables, DWs domain words), search the
// subtrees of open nodes taken from a device queue, depth-first with
// first-fail branching, between the rounds of the fixpoint kernel.
// ---------------------------------------------------------------------------
struct SearchCtr {
    unsigned long long nodes, fails, solutions;
    int32_t maxDepth;
    int32_t nextOpen;    // next open node to hand out
    int32_t nrestQ;      // table restores queued by the decision phase of a round
    int32_t error;       // CT_OK, or why the search stopped (CT_ERR_LEVEL: deeper than the level capacity)
    int32_t started;     // the first decision phase ran
    int32_t cur, round;  // work-list parity to resume a launch with
    int32_t done;        // every slot idle and no open node left (or the node limit reached)
    int32_t pad[2];
};

struct SearchDev {
    int32_t B, T, nv, DWs, maxLevels, segTotal;
    int32_t nopen;
    int32_t roundBudget;          // rounds per launch before it returns (the host launches again)
    long long nodeLimit;          // <= 0: none
    SearchCtr* ctr;
    // per slot
    int32_t* depth;               // [B] frames on the stack
    int32_t* active;              // [B]
    int32_t* busy;                // [B] the slot has tables in the next round (set by the collection)
    int32_t* openIdx;             // [B] open node of the current subtree
    int32_t* depth0;              // [B] tree depth of that open node
    int4* frames;                 // [B][maxLevels] (x, a, branch, -)
    uint32_t* levelDom;           // [B][maxLevels + 1][DWs] domains at each level (level 0: the root)
    int32_t* markAt;              // [B][maxLevels + 1][T] trail position of each table at each level
    int32_t* liveAt;              // [B][maxLevels + 1][T] live chunks of each table at each level
    uint32_t* snapSeg;            // [B][maxLevels + 1][segTotal] index masks of every table at each level
    int32_t* firstOpen;           // [B] open node of the slot's first solution (INT_MAX: none)
    uint32_t* firstSol;           // [B][DWs] the domains of that solution
    int4* restQ;                  // [B * T] queued restores: (slot table j, level, -, -)
    ModelTabCall* calls;          // [B * T] the fixpoint kernel's per-table calls (mark kept current)
    // per model variable and table
    const int32_t* varOff;        // [nv] first domain word of each variable in a slot
    const int32_t* varNW;         // [nv]
    const int32_t* varTabStart;   // [nv + 1] tables of each variable (model table indices)
    const int32_t* varTabList;
    const int32_t* segOff;        // [T] first word of each table's index mask in a level's snapshot
    const int32_t* segTabOf;      // [segTotal] the model table of each word of a level's snapshot
    uint32_t* const* segPtr;      // [B * T] the index masks of every table copy
    // open nodes
    const uint32_t* openDom;      // [nopen][DWs]
    const int32_t* openDepth;     // [nopen]
};

struct ModelDev {
    const TableDev* tabs;       // [ntables]
    const ModelTabCall* calls;  // [ntables]
    const int32_t* scopeBase;   // [ntables + 1] prefix of the arities
    const int32_t* scopeOff;    // word offset of every scope variable in dom
    const int32_t* scopeVar;    // global index of every scope variable
    int32_t* work;              // [2][ntables] work lists (ping-pong by round)
    int32_t* snapTaken;         // [ntables] 1: the table's pending level snapshots were taken in this launch
    int32_t* unitPrefix;        // [ntables + 1] segments of the work list
    int32_t* rowPrefix;         // [ntables + 1] supports rows of the work list
    int32_t* prunedBy;          // [2][nvars] by round parity: -1 none, t one table, -2 several
    ModelCtrl* ctrl;
    uint32_t* dom;
    int32_t* statusBlk;         // mapped host: header, (trail_top, live) per table, domains, node statuses
    int32_t* nodeStatus;        // [ntables / nodeTables] CT_OK or CT_INFEASIBLE per node
    int32_t ntables, nvars, DWg, maxRounds;
    int32_t nodeTables;         // tables per node: node of table t is t / nodeTables
    // Optional prologue of a launch: trail undos done before anything else,
    // and the first round's table count read from device memory.
    const RestoreDesc* restores;  // [nrestores]
    int32_t nrestores;
    const int32_t* nworkIn;     // null: the count is already in ctrl->nwork
    uint64_t* phaseNs;          // null, or [kModelPhases] nanoseconds added per phase (CTA 0's view)
    int4* missQ;                // [sum of the tables' rows] residue misses of a round: (table, row, residue)
    uint32_t spinLimit;         // polls of a grid-barrier wait before it gives up (0: kBarrierSpinLimit)
    SearchDev* search;          // device copy of the search state (search mode only)
};
constexpr int kModelPhases = 8;  // prologue, plan, update, probe, scan, apply, next round, publish
constexpr int kRestoreBatch = 256;
struct RestoreBatch {
    RestoreDesc d[kRestoreBatch];
    int32_t n;
};

// The fixpoint kernel's variant depends on the launch's table count (M.ntables).
int max_coresident_model_blocks(int ntables);
cudaError_t launch_model(const ModelDev& M, int grid, cudaStream_t s);
// The fixpoint kernel in search mode (M.search set): decision and restore
// phases between rounds, until the search is done or the launch's round budget
// is spent. The grid is max_coresident_model_blocks()-bounded as for launch_model.
cudaError_t launch_model_search(const ModelDev& M, int grid, cudaStream_t s);
int max_coresident_search_blocks();
// Level 0 of every slot: the root state of its tables (after a state copy
// into hostTabs), each with an empty trail of trailFactor * W4 + 1024 entries.
cudaError_t launch_search_init(const ModelDev& M, const TableDev* hostTabs, const SearchDev& S,
                               const uint32_t* rootDom, int trailFactor, cudaStream_t s);
cudaError_t launch_restore_batch(const TableDev* tabs, const RestoreBatch& B, cudaStream_t s);
// dst[j] (n clones, j = slot * nsrc + k) takes the state of src[k]: currTable,
// index, residues, lastDom; empty trail (lastpos = -1) and cleared counters.
cudaError_t launch_clone_state(const TableDev* src, const TableDev* dst, int nsrc, int n, cudaStream_t s);

// Launchers (ct_kernels.cu). `dom` is the domain array, `domOff[i]` the word
// offset of scope variable i in it. All run on `s` and return the launch error.
// The propagation kernel is a cooperative launch of `grid` CTAs that must all
// be resident at once (grid <= max_coresident_blocks(variant)).
// variant: bit 0 = every CTA plans in shared memory, bit 1 = batches of 8 rows
// with 3 CTAs per SM (else batches of 16 rows with 2 CTAs per SM).
int max_coresident_blocks(int variant);
cudaError_t launch_propagate(const TableDev& T, int variant, int grid, uint32_t* dom, const int32_t* domOff,
                             const CallParams& P, cudaStream_t s);
cudaError_t launch_save(const TableDev& T, int level, cudaStream_t s);
cudaError_t launch_restore(const TableDev& T, int level, int mark, int top, int newMark, cudaStream_t s);
cudaError_t launch_set_words(uint32_t* dst, const uint32_t* words, int n, cudaStream_t s);
cudaError_t launch_copy_words(uint32_t* dst, const uint32_t* src, int n, cudaStream_t s);
cudaError_t launch_read_ceiling(const uint4* p, size_t n16, cudaStream_t s);

}  // namespace ctk

// Test hook of ct_propagate_noalloc (ct_noalloc.cu): the next call on the
// current device runs its barrier waits out after `polls` polls.
int ct_noalloc_arm_wait_timeout(uint32_t polls);

// Error helpers shared by the host sources (ct_table.cu, ct_model.cu).
void ct_set_error(const char* fmt, ...);
int ct_cuda_fail(cudaError_t e, const char* what);
#define CT_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ct_cuda_fail(e_, #call);   \
    } while (0)

// Internal table entry points used by the model (ct_table.cu).
int ct_table_propagate_on(ct_table* ct, uint32_t* dom, const int32_t* domOffDev, const int32_t* domOffHost,
                          uint32_t* changed, const uint32_t* domHost = nullptr);
const int32_t* ct_table_status_host(const ct_table* ct);
int ct_table_is_empty(const ct_table* ct);
int ct_table_restore_device(ct_table* ct, const ctk::RestoreDesc& d);
// Device memory handed out in 256-byte aligned pieces of one allocation (the
// batched search's table clones); its owner frees it as a whole.
struct DeviceArena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    void* take(size_t bytes) {
        const size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return base + off;
    }
};
// Arena bytes one clone of src takes (dynamic buffers, 8 levels and a trail of
// 2 * W4 + 64 entries, each piece rounded up to 256 bytes).
size_t ct_table_clone_bytes(const ct_table* src);
// A clone of src (see ct_table.cu); its dynamic buffers come from `arena` when
// given (else from cudaMalloc), its Ctrl is `ctrl` when given.
ct_table* ct_table_clone(const ct_table* src, cudaStream_t stream, DeviceArena* arena, ctk::Ctrl* ctrl, int* status);
void ct_table_free(ct_table* ct);
int ct_table_depth(const ct_table* ct);
void ct_table_adopt_state(ct_table* dst, const ct_table* src);
int ct_table_live(const ct_table* ct);
int ct_table_trail_cap(const ct_table* ct);
int ct_table_is_negative(const ct_table* ct);
int ct_table_dom_words(const ct_table* ct);
const int32_t* ct_table_var_ld(const ct_table* ct);
int ct_table_changed_words(const ct_table* ct);
