// ct_internal.cuh -- device layout of a Compact-Table constraint and the
// launchers of its kernels. Private to libct.so.
//
// Device layout of one table (all resident in HBM for the table's lifetime):
//   sup      uint4 [R][W4]   supports rows (Sec. 2, Table 1(b)), value-major:
//                             row jmp[i] + v - lo[i] holds bit j for every
//                             tuple j with tau_j[i] == v; 16-byte aligned rows
//   curr     uint4 [W4]      currTable (Sec. 2, Table 1(c)) as 128-bit chunks
//   idx      int32 [nseg*S]  non-zero index, cut into segments of S chunk
//                             numbers; segment s lists live chunks of the
//                             range [s*S, (s+1)*S) in its first segCnt[s] slots
//   segCnt   int32 [nseg]
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
constexpr int kPlanThreads = 256;
constexpr int kStatusHdr = 16;  // int32 slots before the changed mask
constexpr int kModeDelta = 0;   // mask = ~OR(supports[x, a], a in Delta)
constexpr int kModeReset = 1;   // mask =  OR(supports[x, a], a in dom)
constexpr int32_t kNoChunk = 0x7fffffff;

// Status block header slots (copied to the host after every call).
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
};

// One changed scope variable in the update plan.
struct Group {
    int32_t row_begin;  // first entry in planRows
    int32_t row_count;  // k_i
    int32_t mode;       // kModeDelta / kModeReset
    int32_t var;        // scope position
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
    uint32_t nmiss;      // per call: values whose residue probe missed
    uint32_t done_update;
    uint32_t done_scan;
    int32_t ngroups;
    int32_t nrows;
    int32_t nval, ndelta, nreset, nsup;
    int32_t hits, pruned, trail_added;
    int32_t pad[13];
};

// Everything a kernel needs, passed by value.
struct TableDev {
    const uint4* sup;
    uint4* curr;
    int32_t* idx;
    int32_t* segCnt;
    int32_t* lastpos;
    int2* trailKey;
    uint4* trailOld;
    int32_t* residue;
    uint32_t* lastDom;
    Ctrl* ctrl;
    Group* groups;
    int32_t* planRows;
    int32_t* varSup;
    int32_t* changed;
    int32_t* missRow;
    int32_t* foundChunk;
    const int32_t* rowVar;   // [R] scope position of each row
    const int32_t* varRow0;  // [arity+1] first row of each variable (_supportJmp)
    const int32_t* varNW;    // [arity] words of each domain
    const int32_t* varLD;    // [arity] offset of each domain in lastDom / packed layout
    int32_t* statusBlk;      // [kStatusHdr + nChangedWords + DW]
    int32_t* levelSeg;       // [levelCap][nseg]
    uint32_t* levelDom;      // [levelCap][DW]
    int32_t arity, R, W4, nseg, S, DW, nChangedWords, useResidues;
};

// Launchers (ct_kernels.cu). `dom` is the domain array, `domOff[i]` the word
// offset of scope variable i in it. All run on `s` and return the launch error.
cudaError_t launch_plan(const TableDev& T, const uint32_t* dom, const int32_t* domOff, cudaStream_t s);
cudaError_t launch_update(const TableDev& T, int E, int wpb, const uint32_t* dom, const int32_t* domOff,
                          cudaStream_t s);
cudaError_t launch_scan(const TableDev& T, int E, int wpb, uint32_t* dom, const int32_t* domOff,
                        cudaStream_t s);
cudaError_t launch_save(const TableDev& T, int level, cudaStream_t s);
cudaError_t launch_restore(const TableDev& T, int level, int mark, int top, int newMark, cudaStream_t s);
cudaError_t launch_set_words(uint32_t* dst, const uint32_t* words, int n, cudaStream_t s);
cudaError_t launch_copy_words(uint32_t* dst, const uint32_t* src, int n, cudaStream_t s);

}  // namespace ctk

// Error helpers shared by the host sources (ct_table.cu, ct_model.cu).
void ct_set_error(const char* fmt, ...);
int ct_cuda_fail(cudaError_t e, const char* what);
#define CT_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ct_cuda_fail(e_, #call);   \
    } while (0)

// Internal table entry points used by the model (ct_table.cu).
int ct_table_propagate_on(ct_table* ct, uint32_t* dom, const int32_t* domOffDev, uint32_t* changed);
const int32_t* ct_table_status_host(const ct_table* ct);
int ct_table_dom_words(const ct_table* ct);
const int32_t* ct_table_var_ld(const ct_table* ct);
int ct_table_changed_words(const ct_table* ct);
