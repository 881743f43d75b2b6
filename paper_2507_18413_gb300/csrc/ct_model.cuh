// ct_model.cuh -- the network object shared by the model sources
// (ct_model.cu: fixpoint and depth-first search; ct_search.cu: batched search).
#pragma once
#include <vector>

#include "ct_learn.cuh"
#include "ct_table.cuh"

struct ct_batch;  // the slots of a batched search (ct_search.cu)

struct ct_model {
    int nvars = 0;
    std::vector<int32_t> lo, size, nw, off;
    int DWg = 0;
    uint32_t* d_dom = nullptr;
    std::vector<uint32_t> h_dom;
    std::vector<ct_table*> tables;
    std::vector<std::vector<int>> scopes;
    std::vector<int32_t*> d_tabOff;
    std::vector<std::vector<int32_t>> tabOff;
    std::vector<std::vector<int>> varTables;
    std::vector<char> dirty;
    struct Level {
        std::vector<uint32_t> dom;
        std::vector<char> dirty;
    };
    std::vector<Level> levels;
    uint32_t* h_stage = nullptr;  // pinned staging of the domains (sync_dom)
    bool domStale = false;        // h_dom changed since the device copy was written
    bool domInBlk = false;        // d_dom lives in d_blk
    cudaStream_t stream = nullptr;
    bool ownStream = false;
    ct_options opt{};
    bool staticInfeasible = false;
    bool failed = false;
    int64_t propagations = 0;
    ct_model_stats stats{};  // counters of the one-launch fixpoints
    // the one-launch fixpoint
    bool batch = true;
    bool batchReady = false;
    ctk::ModelDev md{};
    ctk::TableDev* d_tabs = nullptr;
    int32_t* d_blk = nullptr;         // [count, 3 pad | calls[n] | work[2][n]]
    int32_t* h_blk = nullptr;         // pinned mirror of d_blk's head (count, calls, first work list)
    ctk::ModelTabCall* d_calls = nullptr;  // in d_blk
    ctk::ModelTabCall* h_calls = nullptr;  // in h_blk
    int32_t* h_list = nullptr;        // in h_blk: the first round's tables
    int32_t* h_mstatus = nullptr;     // mapped pinned
    std::vector<int> tabVersion;
    std::vector<void*> allocs;
    int grid = 1;
    ct_batch* bsearch = nullptr;  // built by the first batched search, kept for the next ones
    bool hasNegative = false;     // a negative table: no ordering features or lookahead labels
    // learned branching order
    ct_mlp* policy = nullptr;          // NULL: first-fail
    ctk::FeatView* fview = nullptr;    // feature view of the model (one node), built on first use
    int32_t* trace = nullptr;          // branching variables of ct_search_dfs (host)
    int64_t traceCap = 0;
    int64_t* traceCount = nullptr;
};

// Internal helpers of ct_model.cu used by the batched search.
int ct_model_popcount_var(const ct_model* m, int v);
// Replace the domain of variable v (host mirror and device) and schedule its tables.
int ct_model_set_var(ct_model* m, int v, const uint32_t* words);
// Free the batched-search slots of m (ct_search.cu).
void ct_batch_free(ct_batch* b);
// The branching variable of the model's current (propagated) state: the
// policy's best-scored unfixed variable, or first-fail without a policy (or
// when usePolicy is false); -1 when every variable is fixed.
int ct_model_pick_var(ct_model* m, bool usePolicy, int* x);
// Called at every branching node of ct_model_dfs, before the branches.
typedef int (*ct_branch_hook)(void* ctx, ct_model* m);
// The depth-first search of ct_search_dfs with an optional hook.
int ct_model_dfs(ct_model* m, int64_t node_limit, bool countAll, bool usePolicy, ct_search_stats* out,
                 int32_t* first_solution, ct_branch_hook hook, void* ctx);
