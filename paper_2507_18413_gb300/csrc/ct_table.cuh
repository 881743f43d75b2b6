// ct_table.cuh -- the host-side table object, shared by the table, model and
// batched-search sources so that the per-step bookkeeping of thousands of
// table copies (call preparation, results, level pushes and restores) inlines
// into their loops; growth of the device trail and level stack stays out of line.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "ct.h"
#include "ct_internal.cuh"

struct ct_table {
    int arity = 0;
    std::vector<int32_t> lo, size, nw, ld, row0, rowVar;
    int R = 0;
    int64_t t = 0, W = 0, W4 = 0;
    int nseg = 0, S = 32, grid = 1, DW = 0, nChW = 0;
    bool localPlan = true;
    int variant = 1;
    // state read on every call and every step of a batched search, kept together
    int pendingFrom = 0;  // levels [pendingFrom, levels.size()) are not snapshotted yet
    int version = 0;      // bumped when device buffers behind `dev` are reallocated
    int trailTop = 0, trailCap = 0;
    struct Level {
        int mark;  // trail position
        int live;  // live chunks
        int snap;  // snapshot slot: levels saved between two propagations hold one state and
                   // share the lowest one's slot (the one-launch fixpoint writes one snapshot)
    };
    std::vector<Level> levels;    // the saved levels, oldest first
    int live = 0;                 // live chunks of the current state
    int levelCap = 0;
    bool failed = false;
    bool broken = false;  // a device-side wait ran out: the table is unusable
    bool empty = false;
    ctk::TableDev dev{};
    cudaStream_t stream = nullptr;
    bool ownStream = false;
    int32_t* h_status = nullptr;
    size_t statusInts = 0;
    ct_call_stats last{};
    bool profile = false;
    // profile: event pairs around launches, read back lazily (a ring of pairs;
    // the oldest pair is read when the ring is full or the profile is asked for)
    static constexpr int kEvRing = 4096;
    std::vector<cudaEvent_t> ev;  // 2 * kEvRing events, created when profiling is first on
    int evNext = 0, evPending = 0;
    ct_profile prof{};
    int64_t deviceBytes = 0;
    uint32_t* d_domScratch = nullptr;
    std::vector<void*> allocs;
    int64_t shortTuples = 0;     // retained tuples with a wildcard
    bool negative = false;       // the tuples are forbidden
    bool autotuned = false;      // launch shape chosen by trial propagations
    bool copyState = false;      // ablation: currTable round-trips through h_curr every call
    uint32_t* h_curr = nullptr;  // pinned host copy of currTable (copy_state)
    bool trailInArena = false;   // the trail / level stack belong to an arena: not freed here
    bool levelsInArena = false;
    int maxSplit = ctk::kMaxSplit;  // most warps sharing one segment's row list (1: ct_options.no_split)
    bool early = true;              // filter beside the update on calls of few rows (ct_options.no_early_filter)
    uint32_t armPolls = 0;          // test hook: the next call's barrier waits run out after this many polls
};

// Out of line: the device trail grown to hold `need` entries (ct_table.cu).
int ct_table_grow_trail(ct_table* ct, int64_t need);

inline const ctk::TableDev& ct_table_dev(const ct_table* ct) { return ct->dev; }
inline int ct_table_version(const ct_table* ct) { return ct->version; }

// The call of one table in a launch of the one-launch fixpoint: trail room for
// a full update, the newest level's trail mark, the levels pending a snapshot.
inline int ct_table_batch_prepare(ct_table* ct, ctk::ModelTabCall* call) {
    if (ct->broken) {
        ct_set_error("a table is unusable after a device-side timeout");
        return CT_ERR_TIMEOUT;
    }
    if (!ct->levels.empty() && (int64_t)ct->trailTop + ct->W4 > ct->trailCap) {
        const int st = ct_table_grow_trail(ct, (int64_t)ct->trailTop + ct->W4);
        if (st != CT_OK) return st;
    }
    call->mark = ct->levels.empty() ? -1 : ct->levels.back().mark;
    call->snapFrom = ct->pendingFrom;
    call->snapTo = (int)ct->levels.size();
    call->pad = 0;
    return CT_OK;
}

// The launch's results for one table. Levels stay pending until the launch
// that first changes the table, which snapshots them all into the lowest
// one's slot.
inline void ct_table_batch_done(ct_table* ct, int trailTop, int live, bool snapped) {
    ct->trailTop = trailTop;
    if (live > 0) ct->live = live;
    if (snapped) {
        for (int l = ct->pendingFrom; l < (int)ct->levels.size(); ++l) ct->levels[l].snap = ct->pendingFrom;
        ct->pendingFrom = (int)ct->levels.size();
    }
    ct->failed = false;
}

// ct_save on the common path (no failed state, room on the level stack)
// without the call: one level pushed.
inline int ct_table_save_host(ct_table* ct) {
    const int L = (int)ct->levels.size();
    if (ct->failed || (!ct->empty && L + 1 > ct->levelCap)) {
        int lv = 0;
        return ct_save(ct, &lv);
    }
    ct->levels.push_back(ct_table::Level{ct->trailTop, ct->live, L});
    return CT_OK;
}

// Host bookkeeping of a restore; returns 1 (and fills d) when a device undo is needed.
inline int ct_table_restore_prepare(ct_table* ct, int level, ctk::RestoreDesc* d) {
    if (level < 0 || level >= (int)ct->levels.size()) {
        ct_set_error("restore: level %d not in [0, %d)", level, (int)ct->levels.size());
        return CT_ERR_LEVEL;
    }
    if (ct->broken) {
        ct_set_error("restore: the table is unusable after a device-side timeout");
        return CT_ERR_TIMEOUT;
    }
    int need = 0;
    const int mark = ct->levels[level].mark;
    if (!ct->empty && level < ct->pendingFrom) {
        d->level = ct->levels[level].snap;
        d->mark = mark;
        d->top = ct->trailTop;
        ct->trailTop = mark;
        need = 1;
    }
    ct->failed = false;
    ct->live = ct->levels[level].live;
    ct->levels.resize(level);
    ct->pendingFrom = std::min(ct->pendingFrom, level);
    return need;
}
