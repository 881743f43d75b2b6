// ct_learn.cuh -- internal interface of the learned branching order
// (ct_learn.cu): per-variable features of a network's current state, the
// 8 -> 64 -> 64 -> 1 scoring network, and the device views the search drivers
// (ct_model.cu, ct_search.cu) hand to them.
#pragma once
#include <cstdint>
#include <vector>

#include "ct_internal.cuh"

namespace ctk {

constexpr int kNF = 8;    // features per variable
constexpr int kNH = 64;   // hidden units per layer
constexpr int kNW = kNH * kNF + kNH + kNH * kNH + kNH + kNH + 1;  // 4801 weights
constexpr int kTrainBatch = 128;  // largest training batch (one CTA holds it in shared memory)

// A network view for the feature kernels: `nodes` independent copies of a
// network of T tables over V variables (table k of node n is n * T + k,
// variable v of node n is n * V + v).
struct FeatView {
    // static, built once
    int32_t* rowBase = nullptr;   // [nt + 1] prefix of the tables' supports rows
    int32_t* unitBase = nullptr;  // [nt + 1] prefix of segments x scope domain words per table
    int32_t* adjBase = nullptr;   // [nv + 1] tables holding each variable
    int2* adj = nullptr;          // (table, scope position)
    int32_t* varOff = nullptr;    // [nv] word offset of each domain
    int32_t* varNW = nullptr;     // [nv]
    int32_t* varD0 = nullptr;     // [nv] initial domain sizes
    int32_t* deg = nullptr;       // [nv] tables holding each variable
    int32_t* scopeBase = nullptr; // [nt + 1] prefix of the arities
    int32_t* scopeOff = nullptr;  // word offset of every scope variable's domain
    // per call
    uint32_t* counts = nullptr;   // [rowBase[nt]] valid tuples per supports row
    uint32_t* live = nullptr;     // [nt] valid tuples per table
    float* feat = nullptr;        // [nv][kNF]
    float* scores = nullptr;      // [nv]
    float* h_scores = nullptr;    // pinned copy of scores
    int32_t nt = 0, nv = 0, nodes = 1, T = 0, V = 0, degmax = 1, totalUnits = 0, totalRows = 0;
    std::vector<void*> allocs;
};

}  // namespace ctk

struct ct_mlp;  // the scoring network (ct_learn.cu)

// Build the view of `nodes` copies of the network given by the model's scopes
// (per table: scope variables and their word offsets in one node's domain
// array), per-table supports rows and segments, and per-variable domain layout.
int ct_feat_view_build(ctk::FeatView* f, int nodes, const std::vector<std::vector<int>>& scopes,
                       const std::vector<int>& tableR, const std::vector<int>& tableSeg,
                       const std::vector<int32_t>& varOff, const std::vector<int32_t>& varNW,
                       const std::vector<int32_t>& varD0, int DWg);
void ct_feat_view_free(ctk::FeatView* f);
// Features of every variable of the view's nodes (node n only if nodeActive is
// null or nodeActive[n] != 0), from the tables' current currTable and the
// domains in `dom` (device). Stream-ordered; no synchronisation.
int ct_feat_compute(ctk::FeatView* f, const ctk::TableDev* d_tabs, const uint32_t* dom, const uint8_t* nodeActive,
                    cudaStream_t s);
// Scores of the view's variables with the network (after ct_feat_compute),
// copied to f->h_scores; synchronises the stream.
int ct_feat_scores(ctk::FeatView* f, const ct_mlp* mlp, cudaStream_t s);
