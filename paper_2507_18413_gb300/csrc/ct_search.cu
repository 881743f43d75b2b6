// ct_search.cu -- batched depth-first search. The solver of Sec. 4 alternates
// branching and propagation on one node at a time; here many search nodes are
// propagated to their fixpoints together, one cooperative launch per step.
//
// The tree is first expanded on the model itself down to a split depth; the
// nodes met there (open nodes, in depth-first order) are handed to B slots.
// A slot is a copy of the network whose tables share the model's supports
// rows and own their currTable, index, residues, trail and levels; its
// variables and domain words sit in their own range of one domain array. Each
// slot searches its open node's subtree depth-first with the model's
// branching rule (first-fail, left x = min dom x, right x != min dom x). Per
// step the host turns every slot's last result into its next node (branch,
// or backtrack to a level and take the right branch), and one launch of the
// fixpoint kernel first undoes the trails of the backtracking slots, then
// propagates the dirty tables of all slots together; a table failure fails
// only its own slot's node. A slot whose subtree is done takes the next open
// node, or the untried right branch nearest the root of another slot.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ct_model.cuh"

using namespace ctk;

namespace {

struct Frame {
    int x;       // branching variable (model index)
    int a;       // branching value (offset in the initial domain)
    int branch;  // 0: left subtree open, 1: right subtree open, 2: right subtree given to another slot
};

struct OpenNode {
    std::vector<uint32_t> dom;  // domain words before the node's propagation
    int depth;
    std::vector<uint8_t> path;  // branch bits from the root (0 left, 1 right)
};

struct Slot {
    bool active = false;   // exploring a subtree
    bool pending = false;  // its current node is propagated by the next launch
    int depth0 = 0;        // depth of the subtree root
    size_t path0 = 0;      // path length of the subtree root
    std::vector<Frame> stack;
    std::vector<uint32_t> levelDom;  // domain words at each saved level, level-major
    std::vector<uint8_t> path;       // path of the current node
};

// P comes after S in depth-first order without being an ancestor of S.
bool after(const std::vector<uint8_t>& P, const std::vector<uint8_t>& S) {
    const size_t n = std::min(P.size(), S.size());
    for (size_t k = 0; k < n; ++k)
        if (P[k] != S[k]) return P[k] > S[k];
    return false;
}

int popcount_words(const uint32_t* w, int n) {
    int s = 0;
    for (int q = 0; q < n; ++q) s += __builtin_popcount(w[q]);
    return s;
}

// First-fail: the unfixed variable with the smallest domain, ties to the lowest index; -1 if all are fixed.
int first_fail(const ct_model* m, const uint32_t* dom) {
    int x = -1, best = 0;
    for (int v = 0; v < m->nvars; ++v) {
        const int s = popcount_words(dom + m->off[v], m->nw[v]);
        if (s > 1 && (x < 0 || s < best)) {
            x = v;
            best = s;
        }
    }
    return x;
}

int min_value(const ct_model* m, const uint32_t* dom, int v) {
    for (int q = 0; q < m->nw[v]; ++q) {
        const uint32_t w = dom[m->off[v] + q];
        if (w) return q * 32 + __builtin_ctz(w);
    }
    return 0;
}

size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

}  // namespace

struct ct_batch {
    int B = 0, T = 0, n = 0;
    cudaStream_t stream = nullptr;
    std::vector<ct_table*> tabs;  // [n], slot-major: table k of slot s is s * T + k
    TableDev* d_tabs = nullptr;   // [n]
    TableDev* d_src = nullptr;    // [T] the model's own tables, source of the state copies
    std::vector<int> tabVersion;
    // one staging area per step, uploaded with one or two copies:
    // [nwork | calls[n] | dom[B * DWg] | work[2n] | restores[n]]
    char* h_stage = nullptr;  // pinned
    char* d_stage = nullptr;
    size_t offCalls = 0, offDom = 0, offWork = 0, offRest = 0, stageBytes = 0;
    int32_t* h_status = nullptr;  // mapped: header, (trail_top, live) per table, domains, node statuses
    ModelDev md{};
    uint64_t* d_phase = nullptr;  // [kModelPhases] with ct_options.profile
    DeviceArena arena;            // the clones' dynamic buffers (in `allocs`)
    FeatView* fview = nullptr;    // features of the slots (built when a policy is first used)
    uint8_t* d_active = nullptr;  // [B] slots whose features are wanted
    std::vector<uint8_t> h_active;
    int grid = 1;
    std::vector<void*> allocs;
    bool broken = false;
    struct DevSearch* dsearch = nullptr;  // buffers of the search run on the device (built on first use)

    int32_t* nworkHost() { return reinterpret_cast<int32_t*>(h_stage); }
    ModelTabCall* callsHost() { return reinterpret_cast<ModelTabCall*>(h_stage + offCalls); }
    uint32_t* domHost() { return reinterpret_cast<uint32_t*>(h_stage + offDom); }
    int32_t* workHost() { return reinterpret_cast<int32_t*>(h_stage + offWork); }
    RestoreDesc* restHost() { return reinterpret_cast<RestoreDesc*>(h_stage + offRest); }
};

// The search run on the device (ct_search_batch_device): per-slot stacks,
// level records and the open-node queue; the clones' descriptors with their
// own trails (larger than the host-stepped search's, which grows them on the
// host) and control blocks, sharing every other buffer with the clones.
struct DevSearch {
    int B = 0, maxLevels = 0, nopenCap = 0, trailFactor = 0;
    SearchDev hs{};              // device pointers, host copy
    SearchDev* d_sd = nullptr;   // device copy
    TableDev* d_tabs = nullptr;  // [n]
    Ctrl* d_ctrl = nullptr;      // [n]
    uint32_t* d_openDom = nullptr;
    int32_t* d_openDepth = nullptr;
    uint32_t* d_root = nullptr;  // [DWs] root domains
    std::vector<void*> allocs;
};

void dsearch_free(DevSearch* d) {
    if (!d) return;
    for (void* p : d->allocs) cudaFree(p);
    if (d->d_openDom) cudaFree(d->d_openDom);
    if (d->d_openDepth) cudaFree(d->d_openDepth);
    delete d;
}

void ct_batch_free(ct_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    dsearch_free(b->dsearch);
    for (ct_table* t : b->tabs) ct_table_free(t);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->fview) {
        ct_feat_view_free(b->fview);
        delete b->fview;
    }
    cudaGetLastError();
    delete b;
}

namespace {

template <typename T>
int b_alloc(ct_batch* b, T** p, size_t n) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("batched search: cudaMalloc: %s", cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    b->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return CT_OK;
}

// The B copies of the network and the device descriptors of the slot launch.
int build_batch(ct_model* m, int B, ct_batch** out) {
    ct_batch* b = new (std::nothrow) ct_batch();
    if (!b) return CT_ERR_OOM;
    *out = b;
    const int T = (int)m->tables.size();
    const int n = B * T;
    b->B = B;
    b->T = T;
    b->n = n;
    b->stream = m->stream;
    int st = CT_OK;
    // one allocation for every clone's dynamic buffers, first levels and trail,
    // one array for their Ctrl blocks
    size_t perSlot = 0;
    for (int k = 0; k < T; ++k) perSlot += ct_table_clone_bytes(m->tables[k]);
    if ((st = b_alloc(b, &b->arena.base, perSlot * (size_t)B)) != CT_OK) return st;
    b->arena.size = perSlot * (size_t)B;
    Ctrl* dCtrls = nullptr;
    if ((st = b_alloc(b, &dCtrls, (size_t)n)) != CT_OK) return st;
    b->tabs.reserve(n);
    std::vector<Ctrl> hc(n);
    for (int s = 0; s < B; ++s) {
        for (int k = 0; k < T; ++k) {
            const int j = s * T + k;
            ct_table* c = ct_table_clone(m->tables[k], m->stream, &b->arena, dCtrls + j, &st);
            if (!c) return st;
            b->tabs.push_back(c);
            hc[j] = Ctrl{};
            hc[j].cur_mark = -1;
            hc[j].trail_cap = ct_table_trail_cap(c);
        }
    }
    CT_CUDA(cudaMemcpyAsync(dCtrls, hc.data(), (size_t)n * sizeof(Ctrl), cudaMemcpyHostToDevice, m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    const int DWs = B * m->DWg;
    std::vector<int32_t> base(n + 1, 0), off, var;
    for (int s = 0; s < B; ++s) {
        for (int k = 0; k < T; ++k) {
            const int j = s * T + k;
            base[j + 1] = base[j] + (int)m->scopes[k].size();
            for (size_t i = 0; i < m->scopes[k].size(); ++i) {
                off.push_back(m->tabOff[k][i] + s * m->DWg);
                var.push_back(m->scopes[k][i] + s * m->nvars);
            }
        }
    }
    int32_t *dBase, *dOff, *dVar, *dPruned, *dNode, *dUnit, *dRow, *dSnap;
    ModelCtrl* dCtrl;
    if (m->opt.profile && (st = b_alloc(b, &b->d_phase, kModelPhases)) != CT_OK) return st;
    if ((st = b_alloc(b, &b->d_tabs, n)) != CT_OK || (st = b_alloc(b, &b->d_src, T)) != CT_OK ||
        (st = b_alloc(b, &dBase, n + 1)) != CT_OK || (st = b_alloc(b, &dOff, off.size())) != CT_OK ||
        (st = b_alloc(b, &dVar, var.size())) != CT_OK || (st = b_alloc(b, &dPruned, 2 * (size_t)B * m->nvars)) != CT_OK ||
        (st = b_alloc(b, &dNode, B)) != CT_OK || (st = b_alloc(b, &dUnit, n + 1)) != CT_OK ||
        (st = b_alloc(b, &dRow, n + 1)) != CT_OK || (st = b_alloc(b, &dCtrl, 1)) != CT_OK ||
        (st = b_alloc(b, &dSnap, n)) != CT_OK)
        return st;
    b->offCalls = 16;
    b->offDom = align16(b->offCalls + (size_t)n * sizeof(ModelTabCall));
    b->offWork = align16(b->offDom + (size_t)DWs * sizeof(uint32_t));
    b->offRest = align16(b->offWork + 2 * (size_t)n * sizeof(int32_t));
    b->stageBytes = align16(b->offRest + (size_t)n * sizeof(RestoreDesc));
    if ((st = b_alloc(b, &b->d_stage, b->stageBytes)) != CT_OK) return st;
    const size_t statusInts = (size_t)kModelHdr + 2 * (size_t)n + DWs + B + n;
    if (cudaHostAlloc((void**)&b->h_stage, b->stageBytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&b->h_status, statusInts * sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("batched search: pinned host buffers");
        return CT_ERR_OOM;
    }
    std::memset(b->h_stage, 0, b->stageBytes);
    int32_t* dStatus = nullptr;
    CT_CUDA(cudaHostGetDevicePointer((void**)&dStatus, b->h_status, 0));
    cudaStream_t s = m->stream;
    CT_CUDA(cudaMemcpyAsync(dBase, base.data(), base.size() * 4, cudaMemcpyHostToDevice, s));
    CT_CUDA(cudaMemcpyAsync(dOff, off.data(), off.size() * 4, cudaMemcpyHostToDevice, s));
    CT_CUDA(cudaMemcpyAsync(dVar, var.data(), var.size() * 4, cudaMemcpyHostToDevice, s));
    CT_CUDA(cudaMemsetAsync(dPruned, 0xff, 2 * (size_t)B * m->nvars * 4, s));
    CT_CUDA(cudaMemsetAsync(dNode, 0, (size_t)B * 4, s));
    CT_CUDA(cudaMemsetAsync(dCtrl, 0, sizeof(ModelCtrl), s));
    CT_CUDA(cudaMemsetAsync(dSnap, 0, (size_t)n * sizeof(int32_t), s));
    std::vector<TableDev> td(n);
    b->tabVersion.resize(n);
    for (int j = 0; j < n; ++j) {
        td[j] = ct_table_dev(b->tabs[j]);
        b->tabVersion[j] = ct_table_version(b->tabs[j]);
    }
    CT_CUDA(cudaMemcpyAsync(b->d_tabs, td.data(), (size_t)n * sizeof(TableDev), cudaMemcpyHostToDevice, s));
    CT_CUDA(cudaStreamSynchronize(s));  // td and the host vectors above go out of scope
    ModelDev& M = b->md;
    M.tabs = b->d_tabs;
    M.calls = reinterpret_cast<const ModelTabCall*>(b->d_stage + b->offCalls);
    M.scopeBase = dBase;
    M.scopeOff = dOff;
    M.scopeVar = dVar;
    M.work = reinterpret_cast<int32_t*>(b->d_stage + b->offWork);
    M.unitPrefix = dUnit;
    M.rowPrefix = dRow;
    M.prunedBy = dPruned;
    M.ctrl = dCtrl;
    M.snapTaken = dSnap;
    M.dom = reinterpret_cast<uint32_t*>(b->d_stage + b->offDom);
    M.statusBlk = dStatus;
    M.nodeStatus = dNode;
    M.ntables = n;
    M.nvars = B * m->nvars;
    M.DWg = DWs;
    int64_t domBits = 0;
    for (int v = 0; v < m->nvars; ++v) domBits += m->size[v];
    M.maxRounds = (int)std::min<int64_t>(domBits + 2, 1 << 30);
    M.nodeTables = T;
    M.restores = reinterpret_cast<const RestoreDesc*>(b->d_stage + b->offRest);
    M.nrestores = 0;
    M.nworkIn = reinterpret_cast<const int32_t*>(b->d_stage);
    M.phaseNs = b->d_phase;
    const int maxCo = max_coresident_model_blocks(n);
    if (maxCo <= 0) {
        ct_set_error("batched search: the fixpoint kernel cannot be made resident on this device");
        return CT_ERR_CUDA;
    }
    int64_t segs = 0, rows = 0;
    for (ct_table* tab : m->tables) {
        segs += ct_table_dev(tab).nseg;
        rows += ct_table_dev(tab).R;
    }
    if ((st = b_alloc(b, &M.missQ, (size_t)std::max<int64_t>(B * rows, 1))) != CT_OK) return st;
    int64_t want = std::max<int64_t>({(int64_t)n, B * ((segs + kWarps - 1) / kWarps),
                                      B * ((rows + 2 * kWarps - 1) / (2 * kWarps)), 1});
    if (m->opt.grid_blocks > 0) want = m->opt.grid_blocks;
    b->grid = (int)std::min<int64_t>(want, maxCo);
    return CT_OK;
}

// The feature view of the B slots (for a policy).
int ensure_slot_features(ct_model* m, ct_batch* b) {
    if (b->fview) return CT_OK;
    const int T = b->T;
    std::vector<int> R(T), seg(T);
    for (int k = 0; k < T; ++k) {
        R[k] = ct_table_dev(m->tables[k]).R;
        seg[k] = ct_table_dev(m->tables[k]).nseg;
    }
    FeatView* f = new (std::nothrow) FeatView();
    if (!f) return CT_ERR_OOM;
    int st = ct_feat_view_build(f, b->B, m->scopes, R, seg, m->off, m->nw, m->size, m->DWg);
    if (st == CT_OK) st = b_alloc(b, &b->d_active, b->B);
    if (st != CT_OK) {
        ct_feat_view_free(f);
        delete f;
        return st;
    }
    b->fview = f;
    b->h_active.assign(b->B, 0);
    return CT_OK;
}

// Every copy takes the current state of the model's tables (one launch).
int sync_copies(ct_model* m, ct_batch* b) {
    std::vector<TableDev> td(b->T);
    for (int k = 0; k < b->T; ++k) td[k] = ct_table_dev(m->tables[k]);
    CT_CUDA(cudaMemcpyAsync(b->d_src, td.data(), td.size() * sizeof(TableDev), cudaMemcpyHostToDevice, b->stream));
    CT_CUDA(launch_clone_state(b->d_src, b->d_tabs, b->T, b->n, b->stream));
    CT_CUDA(cudaStreamSynchronize(b->stream));
    for (int j = 0; j < b->n; ++j) ct_table_adopt_state(b->tabs[j], m->tables[j % b->T]);
    return CT_OK;
}

template <typename T>
int d_alloc(DevSearch* d, T** p, size_t n) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("device search: cudaMalloc of %zu bytes: %s", std::max<size_t>(n, 1) * sizeof(T),
                     cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    d->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return CT_OK;
}

// First capacities of the device search, doubled (up to the maxima) and the
// search run again when a subtree needs more.
constexpr int kDevLevels = 64, kDevLevelsMax = 1024;        // levels below an open node
constexpr int kDevTrailFactor = 16, kDevTrailFactorMax = 128;  // trail entries per table: factor x chunks + 1024
constexpr int kDevRoundBudget = 1024;  // rounds per launch
constexpr int kDevOpenPerSlot = 2;      // the device search splits until this many open nodes per slot
constexpr int kMaxSplitDepth = 48;      // ... or this depth

// The device search's buffers for the B slots of b (kept with b).
int build_dsearch(ct_model* m, ct_batch* b, int levels, int trailFactor, DevSearch** out) {
    DevSearch* d = new (std::nothrow) DevSearch();
    if (!d) return CT_ERR_OOM;
    *out = d;
    const int B = b->B, T = b->T, n = b->n, DWs = m->DWg, nv = m->nvars, L = levels;
    d->B = B;
    d->maxLevels = L;
    d->trailFactor = trailFactor;
    std::vector<int32_t> segOff(T + 1, 0), varTabStart(nv + 1, 0), varTabList;
    for (int k = 0; k < T; ++k) segOff[k + 1] = segOff[k] + ct_table_dev(m->tables[k]).nseg;
    for (int v = 0; v < nv; ++v) {
        for (int k : m->varTables[v]) varTabList.push_back(k);
        varTabStart[v + 1] = (int32_t)varTabList.size();
    }
    SearchDev& S = d->hs;
    S.B = B;
    S.T = T;
    S.nv = nv;
    S.DWs = DWs;
    S.maxLevels = L;
    S.segTotal = segOff[T];
    S.roundBudget = kDevRoundBudget;
    const size_t lv = (size_t)B * (L + 1);
    int st = CT_OK;
    int32_t *vOff, *vNW, *vTS, *vTL, *sOff, *sTab;
    uint32_t** sPtr;
    if ((st = d_alloc(d, &S.ctr, 1)) || (st = d_alloc(d, &S.depth, B)) || (st = d_alloc(d, &S.active, B)) ||
        (st = d_alloc(d, &S.busy, B)) || (st = d_alloc(d, &S.openIdx, B)) || (st = d_alloc(d, &S.depth0, B)) ||
        (st = d_alloc(d, &S.frames, (size_t)B * L)) || (st = d_alloc(d, &S.levelDom, lv * DWs)) ||
        (st = d_alloc(d, &S.markAt, lv * T)) || (st = d_alloc(d, &S.liveAt, lv * T)) ||
        (st = d_alloc(d, &S.snapSeg, lv * S.segTotal)) || (st = d_alloc(d, &S.firstOpen, B)) ||
        (st = d_alloc(d, &S.firstSol, (size_t)B * DWs)) || (st = d_alloc(d, &S.restQ, (size_t)n)) ||
        (st = d_alloc(d, &vOff, nv)) || (st = d_alloc(d, &vNW, nv)) || (st = d_alloc(d, &vTS, nv + 1)) ||
        (st = d_alloc(d, &vTL, varTabList.size())) || (st = d_alloc(d, &sOff, T + 1)) ||
        (st = d_alloc(d, &sTab, S.segTotal)) || (st = d_alloc(d, &sPtr, (size_t)n)) ||
        (st = d_alloc(d, &d->d_sd, 1)) || (st = d_alloc(d, &d->d_tabs, n)) || (st = d_alloc(d, &d->d_ctrl, n)) ||
        (st = d_alloc(d, &d->d_root, DWs)))
        return st;
    S.calls = reinterpret_cast<ModelTabCall*>(b->d_stage + b->offCalls);
    S.varOff = vOff;
    S.varNW = vNW;
    S.varTabStart = vTS;
    S.varTabList = vTL;
    S.segOff = sOff;
    S.segTabOf = sTab;
    S.segPtr = sPtr;
    std::vector<int32_t> segTab(S.segTotal);
    for (int k = 0; k < T; ++k)
        for (int q = segOff[k]; q < segOff[k + 1]; ++q) segTab[q] = k;
    std::vector<uint32_t*> segPtrs(n);
    for (int j = 0; j < n; ++j) segPtrs[j] = ct_table_dev(b->tabs[j]).segMask;
    cudaStream_t str = b->stream;
    if (S.segTotal > 0)
        CT_CUDA(cudaMemcpyAsync(sTab, segTab.data(), segTab.size() * 4, cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaMemcpyAsync(sPtr, segPtrs.data(), n * sizeof(uint32_t*), cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaMemcpyAsync(vOff, m->off.data(), nv * 4, cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaMemcpyAsync(vNW, m->nw.data(), nv * 4, cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaMemcpyAsync(vTS, varTabStart.data(), (nv + 1) * 4, cudaMemcpyHostToDevice, str));
    if (!varTabList.empty())
        CT_CUDA(cudaMemcpyAsync(vTL, varTabList.data(), varTabList.size() * 4, cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaMemcpyAsync(sOff, segOff.data(), (T + 1) * 4, cudaMemcpyHostToDevice, str));
    // the clones' descriptors with their own trails and control blocks
    std::vector<TableDev> td(n);
    size_t entries = 0;
    for (int j = 0; j < n; ++j) entries += (size_t)trailFactor * ct_table_dev(b->tabs[j]).W4 + 1024;
    int2* keys = nullptr;
    uint4* olds = nullptr;
    if ((st = d_alloc(d, &keys, entries)) || (st = d_alloc(d, &olds, entries))) return st;
    size_t at = 0;
    for (int j = 0; j < n; ++j) {
        td[j] = ct_table_dev(b->tabs[j]);
        td[j].trailKey = keys + at;
        td[j].trailOld = olds + at;
        td[j].ctrl = d->d_ctrl + j;
        at += (size_t)trailFactor * td[j].W4 + 1024;
    }
    CT_CUDA(cudaMemcpyAsync(d->d_tabs, td.data(), n * sizeof(TableDev), cudaMemcpyHostToDevice, str));
    CT_CUDA(cudaStreamSynchronize(str));  // the host vectors above go out of scope
    return CT_OK;
}

struct Search {
    ct_model* m = nullptr;
    ct_batch* b = nullptr;
    int B = 0, splitDepth = 0;
    bool splitAssign = false;  // splitDepth counts assignments (left branches) on a node's path
    int64_t minOpen = 0;       // the breadth-first split goes on below splitDepth while fewer open nodes
    int64_t limit = 0;
    bool countAll = true;
    bool anyStop = false;  // stop at the first solution any slot finds
    ct_search_stats st{};
    ct_batch_info info{};
    bool hitLimit = false;
    bool stopIssue = false;  // no new node is started (node limit)
    bool splitStop = false;  // the split phase found the first solution it was asked for
    int64_t splitBudget = 0;   // > 0: the model's share of nodes before the slots take over
    bool budgetHit = false;
    bool haveBest = false;
    std::vector<uint8_t> bestPath;
    std::vector<int32_t> bestVals;
    std::vector<OpenNode> open;
    size_t nextOpen = 0;
    std::vector<uint32_t> rootDom;
    bool copiesReady = false;
    std::vector<Slot> slots;
    std::vector<char> dirty;       // [n]
    std::vector<int> restPos;      // [n] index in this step's restore list, -1 none
    int nrest = 0;
    bool usePolicy = false;        // branch with the model's policy (scores of the slots per step)
    const float* scores = nullptr; // this step's scores of the slots' variables
    // lookahead probes instead of a search: per slot, the label of its probe
    bool probeMode = false;
    double probeL = 0.0;
    std::vector<float> probeLabel;
    // breadth-first split: per slot, the result of the node it propagated
    struct SplitOut {
        int status = CT_OK;
        int x = -1;  // branching variable, -1: a solution
        std::vector<uint32_t> dom;
    };
    bool splitMode = false;
    bool slotsReady = false;
    std::vector<SplitOut> splitOut;
    std::chrono::steady_clock::time_point t0;

    uint32_t* slotDom(int s) { return b->domHost() + (size_t)s * m->DWg; }
    const uint32_t* slotDom(int s) const { return b->domHost() + (size_t)s * m->DWg; }

    void record_solution(const std::vector<uint8_t>& path, const uint32_t* dom) {
        st.solutions += 1;
        if (haveBest && !after(bestPath, path)) return;
        haveBest = true;
        bestPath = path;
        bestVals.resize(m->nvars);
        for (int v = 0; v < m->nvars; ++v) bestVals[v] = m->lo[v] + min_value(m, dom, v);
    }

    int ensure_copies() {
        const auto c0 = std::chrono::steady_clock::now();
        int rc;
        if (b && (b->B != B || b->broken)) {
            ct_batch_free(b);
            b = m->bsearch = nullptr;
        }
        if (!b) {
            ct_batch* nb = nullptr;
            rc = build_batch(m, B, &nb);
            if (rc != CT_OK) {
                ct_batch_free(nb);
                return rc;
            }
            b = m->bsearch = nb;
        }
        if ((rc = sync_copies(m, b)) != CT_OK) {
            b->broken = true;
            return rc;
        }
        rootDom = m->h_dom;
        copiesReady = true;
        info.setup_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
        return CT_OK;
    }

    // ---- split phase: depth-first on the model itself ----
    int split(int depth, std::vector<uint8_t>& path) {
        if (depth == splitDepth || budgetHit) {
            open.push_back(OpenNode{m->h_dom, depth, path});
            return CT_OK;
        }
        if (splitBudget > 0 && info.split_nodes >= splitBudget) {
            // the model searched its share: this node and every untried right
            // branch above it (recorded on the way back) go to the slots
            budgetHit = true;
            open.push_back(OpenNode{m->h_dom, depth, path});
            return CT_OK;
        }
        if (limit > 0 && st.nodes >= limit) {
            hitLimit = stopIssue = true;
            return CT_OK;
        }
        st.nodes += 1;
        info.split_nodes += 1;
        if (depth > st.max_depth) st.max_depth = depth;
        int r = ct_model_propagate(m);
        if (r < 0) return r;
        if (r == CT_INFEASIBLE) {
            st.fails += 1;
            return CT_OK;
        }
        int x = -1;
        if ((r = ct_model_pick_var(m, usePolicy, &x)) != CT_OK) return r;
        if (x < 0) {
            record_solution(path, m->h_dom.data());
            if (!countAll) splitStop = true;
            return CT_OK;
        }
        const int a = min_value(m, m->h_dom.data(), x);
        const int nwx = m->nw[x];
        std::vector<uint32_t> left(nwx, 0u), right(m->h_dom.begin() + m->off[x], m->h_dom.begin() + m->off[x] + nwx);
        left[a >> 5] = 1u << (a & 31);
        right[a >> 5] &= ~(1u << (a & 31));
        for (int br = 0; br < 2; ++br) {
            if (br == 1 && budgetHit) {
                std::vector<uint32_t> dom = m->h_dom;
                std::copy(right.begin(), right.end(), dom.begin() + m->off[x]);
                path.push_back(1);
                open.push_back(OpenNode{std::move(dom), depth + 1, path});
                path.pop_back();
                break;
            }
            int L = 0;
            int rc = ct_model_save(m, &L);
            if (rc != CT_OK) return rc;
            rc = ct_model_set_var(m, x, br == 0 ? left.data() : right.data());
            path.push_back((uint8_t)br);
            if (rc == CT_OK) rc = split(depth + 1, path);
            path.pop_back();
            const int rr = ct_model_restore(m, L);
            if (rc != CT_OK) return rc;
            if (rr != CT_OK) return rr;
            if (stopIssue || splitStop) break;
        }
        // Back at the root fixpoint: the slot copies take this state, only when
        // open nodes are left for them.
        if (depth == 0 && !open.empty() && !copiesReady) return ensure_copies();
        return CT_OK;
    }

    // ---- split phase, breadth-first in the slots ----
    // The root is propagated on the model; then every level of the tree above
    // the split depth is propagated together, up to B nodes per launch, each
    // node in a slot from the root state (the slot is put back at the root
    // afterwards, its undo staged for the next launch). Children are made in
    // the order of their parents, left before right, so each level, and the
    // open nodes left at the split depth, stay in depth-first order. The nodes
    // visited are those of the depth-first split.
    void children(std::vector<OpenNode>& out, const std::vector<uint32_t>& dom, int x, int depth,
                  const std::vector<uint8_t>& path) {
        const int a = min_value(m, dom.data(), x);
        for (int br = 0; br < 2; ++br) {
            OpenNode c{dom, depth, path};
            uint32_t* w = c.dom.data() + m->off[x];
            if (br == 0) {
                for (int q = 0; q < m->nw[x]; ++q) w[q] = 0u;
                w[a >> 5] = 1u << (a & 31);
            } else {
                w[a >> 5] &= ~(1u << (a & 31));
            }
            c.path.push_back((uint8_t)br);
            if (!countAll && haveBest && after(c.path, bestPath)) continue;
            out.push_back(std::move(c));
        }
    }

    int split_bfs() {
        if (limit > 0 && st.nodes >= limit) {
            hitLimit = stopIssue = true;
            return CT_OK;
        }
        st.nodes += 1;
        info.split_nodes += 1;
        int r = ct_model_propagate(m);
        if (r < 0) return r;
        if (r == CT_INFEASIBLE) {
            st.fails += 1;
            return CT_OK;
        }
        int x = -1;
        if ((r = ct_model_pick_var(m, usePolicy, &x)) != CT_OK) return r;
        if (x < 0) {
            record_solution(std::vector<uint8_t>(), m->h_dom.data());
            return CT_OK;
        }
        if ((r = ensure_copies()) != CT_OK) return r;
        if (usePolicy && (r = ensure_slot_features(m, b)) != CT_OK) return r;
        init_slots();
        splitOut.assign(B, SplitOut());
        std::vector<OpenNode> F, G;
        children(F, m->h_dom, x, 1, std::vector<uint8_t>());
        for (int depth = 1; !F.empty() && !stopIssue; ++depth) {
            if (!splitAssign && depth >= splitDepth && ((int64_t)F.size() >= minOpen || depth >= kMaxSplitDepth))
                break;
            if (splitAssign) {
                // nodes with splitDepth assignments on their path are open nodes
                std::vector<OpenNode> rest;
                for (OpenNode& o : F) {
                    int a = 0;
                    for (uint8_t br : o.path) a += br == 0;
                    if (a >= splitDepth) open.push_back(std::move(o));
                    else rest.push_back(std::move(o));
                }
                F.swap(rest);
                if (F.empty()) break;
            }
            G.clear();
            for (size_t i0 = 0; i0 < F.size() && !stopIssue; i0 += (size_t)B) {
                const size_t i1 = std::min(F.size(), i0 + (size_t)B);
                splitMode = true;
                bool any = false;
                for (size_t i = i0; i < i1 && !stopIssue; ++i) {
                    if (!countAll && haveBest && after(F[i].path, bestPath)) continue;
                    const int s = (int)(i - i0);
                    if ((r = start(s, F[i].dom.data(), F[i].depth, F[i].path)) != CT_OK) return r;
                    any |= slots[s].pending;
                }
                if (any) r = step();
                splitMode = false;
                if (r != CT_OK) return r;
                if (!any) break;
                for (size_t i = i0; i < i1; ++i) {
                    const int s = (int)(i - i0);
                    if (slots[s].pending) continue;  // never issued
                    SplitOut& o = splitOut[s];
                    if (o.dom.empty()) continue;
                    if (o.status != CT_OK) st.fails += 1;
                    else if (o.x < 0) record_solution(F[i].path, o.dom.data());
                    else children(G, o.dom, o.x, depth + 1, F[i].path);
                    o.dom.clear();
                }
            }
            F.swap(G);
        }
        for (OpenNode& o : F) open.push_back(std::move(o));
        if (splitAssign) {
            // open nodes met at different tree depths, put in depth-first order:
            // no open node is an ancestor of another, so that is the
            // lexicographic order of the paths (left before right)
            std::sort(open.begin(), open.end(), [](const OpenNode& a, const OpenNode& b) {
                return std::lexicographical_compare(a.path.begin(), a.path.end(), b.path.begin(), b.path.end());
            });
        }
        return CT_OK;
    }

    // ---- slot bookkeeping ----
    void mark_var(int s, int v) {
        for (int k : m->varTables[v]) dirty[(size_t)s * b->T + k] = 1;
    }

    int save_slot(int s) {
        Slot& S = slots[s];
        for (int k = 0; k < b->T; ++k) {
            const int rc = ct_table_save_host(b->tabs[(size_t)s * b->T + k]);
            if (rc != CT_OK) return rc;
        }
        const uint32_t* d = slotDom(s);
        S.levelDom.insert(S.levelDom.end(), d, d + m->DWg);
        return CT_OK;
    }

    // Back to saved level L: trails undone by the next launch (one undo per
    // table and step, from the lowest level asked for), domains from the host copy.
    int restore_slot(int s, int L) {
        Slot& S = slots[s];
        for (int k = 0; k < b->T; ++k) {
            const int j = s * b->T + k;
            RestoreDesc d{};
            const int need = ct_table_restore_prepare(b->tabs[j], L, &d);
            if (need < 0) return need;
            if (!need) continue;
            d.table = j;
            RestoreDesc* R = b->restHost();
            if (restPos[j] >= 0) {
                RestoreDesc& e = R[restPos[j]];  // an earlier undo of this step: extend it down to level L
                e.level = d.level;
                e.mark = d.mark;
            } else {
                restPos[j] = nrest;
                R[nrest++] = d;
            }
        }
        std::memcpy(slotDom(s), S.levelDom.data() + (size_t)L * m->DWg, (size_t)m->DWg * sizeof(uint32_t));
        S.levelDom.resize((size_t)L * m->DWg);
        return CT_OK;
    }

    int cancel(int s) {
        Slot& S = slots[s];
        const int rc = S.active ? restore_slot(s, 0) : CT_OK;
        S.active = false;
        S.pending = false;
        S.stack.clear();
        S.path.clear();
        return rc;
    }

    // The slot's current node goes into the next launch.
    int issue(int s, int depth) {
        if (anyStop && haveBest) return cancel(s);
        if (limit > 0 && st.nodes >= limit) {
            hitLimit = stopIssue = true;
            return cancel(s);
        }
        st.nodes += 1;
        if (splitMode) info.split_nodes += 1;
        else info.slot_nodes += 1;
        if (depth > st.max_depth) st.max_depth = depth;
        slots[s].pending = true;
        return CT_OK;
    }

    int start(int s, const uint32_t* dom, int depth, const std::vector<uint8_t>& path) {
        Slot& S = slots[s];
        int rc = save_slot(s);  // level 0: the root state
        if (rc != CT_OK) return rc;
        std::memcpy(slotDom(s), dom, (size_t)m->DWg * sizeof(uint32_t));
        for (int k = 0; k < b->T; ++k) dirty[(size_t)s * b->T + k] = 1;
        S.active = true;
        S.depth0 = depth;
        S.stack.clear();
        S.path = path;
        S.path0 = path.size();
        return issue(s, depth);
    }

    // An idle slot takes the next open node, else the untried right branch
    // nearest the root among the other slots' subtrees.
    int assign(int s) {
        if (anyStop && haveBest) return CT_OK;
        while (!stopIssue && nextOpen < open.size()) {
            const OpenNode& o = open[nextOpen++];
            if (!countAll && haveBest && after(o.path, bestPath)) continue;
            info.open_nodes += 1;
            return start(s, o.dom.data(), o.depth, o.path);
        }
        if (stopIssue) return CT_OK;
        int v = -1, fj = -1, bestDepth = 0;
        for (int u = 0; u < B; ++u) {
            const Slot& U = slots[u];
            if (!U.active) continue;
            for (int j = 0; j < (int)U.stack.size(); ++j) {
                if (U.stack[j].branch != 0) continue;
                if (v < 0 || U.depth0 + j < bestDepth) {
                    v = u;
                    fj = j;
                    bestDepth = U.depth0 + j;
                }
                break;  // deeper frames of this slot are further from the root
            }
        }
        if (v < 0) return CT_OK;
        Slot& V = slots[v];
        std::vector<uint8_t> path(V.path.begin(), V.path.begin() + (V.path0 + fj));
        path.push_back(1);
        if (!countAll && haveBest && after(path, bestPath)) return CT_OK;
        Frame& f = V.stack[fj];
        f.branch = 2;
        std::vector<uint32_t> dom(V.levelDom.begin() + (size_t)(fj + 1) * m->DWg,
                                  V.levelDom.begin() + (size_t)(fj + 2) * m->DWg);
        dom[m->off[f.x] + (f.a >> 5)] &= ~(1u << (f.a & 31));
        info.steals += 1;
        return start(s, dom.data(), V.depth0 + fj + 1, path);
    }

    int branch(int s, int x) {
        Slot& S = slots[s];
        uint32_t* dom = slotDom(s);
        const int a = min_value(m, dom, x);
        int rc = save_slot(s);  // level stack.size() + 1
        if (rc != CT_OK) return rc;
        S.stack.push_back(Frame{x, a, 0});
        for (int q = 0; q < m->nw[x]; ++q) dom[m->off[x] + q] = 0u;
        dom[m->off[x] + (a >> 5)] = 1u << (a & 31);
        mark_var(s, x);
        S.path.push_back(0);
        return issue(s, S.depth0 + (int)S.stack.size());
    }

    int backtrack(int s) {
        Slot& S = slots[s];
        while (!S.stack.empty()) {
            const int j = (int)S.stack.size() - 1;
            Frame& f = S.stack[j];
            int rc = restore_slot(s, j + 1);
            if (rc != CT_OK) return rc;
            S.path.resize(S.path0 + j);
            if (f.branch == 0) {
                f.branch = 1;
                S.path.push_back(1);
                if (!countAll && haveBest && after(S.path, bestPath)) return cancel(s);
                if ((rc = save_slot(s)) != CT_OK) return rc;
                uint32_t* dom = slotDom(s);
                dom[m->off[f.x] + (f.a >> 5)] &= ~(1u << (f.a & 31));
                mark_var(s, f.x);
                return issue(s, S.depth0 + j + 1);
            }
            S.stack.pop_back();
        }
        return cancel(s);  // subtree done: back to the root state, idle
    }

    // Branching variable of slot s's propagated node (the policy's best score
    // or first-fail); -1 when every variable is fixed.
    int pick(int s) const {
        int x = -1;
        const uint32_t* dom = slotDom(s);
        if (scores) {
            const float* sc = scores + (size_t)s * m->nvars;
            for (int v = 0; v < m->nvars; ++v)
                if (popcount_words(dom + m->off[v], m->nw[v]) > 1 && (x < 0 || sc[v] > sc[x])) x = v;
        } else {
            x = first_fail(m, dom);
        }
        return x;
    }

    // The result of slot s's node (status of its fixpoint, domains in slotDom).
    int advance(int s, int nodeStatus) {
        Slot& S = slots[s];
        S.pending = false;
        if (!countAll && haveBest && after(S.path, bestPath)) return cancel(s);
        if (nodeStatus == CT_INFEASIBLE) {
            st.fails += 1;
            return backtrack(s);
        }
        const int x = pick(s);
        if (x < 0) {
            record_solution(S.path, slotDom(s));
            return backtrack(s);
        }
        return branch(s, x);
    }

    // One launch: undo the trails of this step, propagate the dirty tables of every slot.
    int step() {
        const int n = b->n, T = b->T;
        int32_t* work = b->workHost();
        int nwork = 0;
        for (int j = 0; j < n; ++j)
            if (dirty[j]) work[nwork++] = j;
        info.steps += 1;
        if (nwork == 0 && nrest == 0 && !usePolicy && !probeMode && !splitMode) {  // the nodes are their own fixpoints
            std::vector<int> ps;
            for (int s = 0; s < B; ++s)
                if (slots[s].pending) ps.push_back(s);
            for (int s : ps) {
                const int rc = advance(s, CT_OK);
                if (rc != CT_OK) return rc;
            }
            return CT_OK;
        }
        int rc;
        // per table, one visit: its call (trail room, mark, pending level
        // snapshots) and, when its buffers moved, its device descriptor
        ModelTabCall* calls = b->callsHost();
        for (int j = 0; j < n; ++j) {
            if ((rc = ct_table_batch_prepare(b->tabs[j], &calls[j])) != CT_OK) return rc;
            const int v = ct_table_version(b->tabs[j]);
            if (v != b->tabVersion[j]) {
                CT_CUDA(cudaMemcpyAsync(b->d_tabs + j, &ct_table_dev(b->tabs[j]), sizeof(TableDev),
                                        cudaMemcpyHostToDevice, b->stream));
                b->tabVersion[j] = v;
            }
        }
        b->nworkHost()[0] = nwork;
        CT_CUDA(cudaMemcpyAsync(b->d_stage, b->h_stage, b->offWork + (size_t)nwork * sizeof(int32_t),
                                cudaMemcpyHostToDevice, b->stream));
        if (nrest > 0)
            CT_CUDA(cudaMemcpyAsync(b->d_stage + b->offRest, b->h_stage + b->offRest,
                                    (size_t)nrest * sizeof(RestoreDesc), cudaMemcpyHostToDevice, b->stream));
        b->md.nrestores = nrest;
        volatile int32_t* H = b->h_status;
        H[0] = kNoChunk;
        const auto w0 = std::chrono::steady_clock::now();
        CT_CUDA(launch_model(b->md, b->grid, b->stream));
        bool seen = false;
        for (uint64_t it = 0;; ++it) {
            if (H[0] != kNoChunk) {
                seen = true;
                break;
            }
            if ((it & 1023u) == 1023u && std::chrono::steady_clock::now() - w0 > std::chrono::milliseconds(kHostWaitMs))
                break;
        }
        if (!seen) CT_CUDA(cudaStreamSynchronize(b->stream));
        info.wait_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - w0).count();
        const int status = H[0];
        if (status != CT_OK) {
            b->broken = true;
            if (status == kNoChunk) {
                ct_set_error("batched search: the fixpoint kernel did not publish (a device-side wait ran out)");
                return CT_ERR_TIMEOUT;
            }
            ct_set_error("batched search: fixpoint kernel status %d", status);
            return status < 0 ? status : CT_ERR_STATE;
        }
        st.propagations += H[2];
        info.rounds += H[1];
        info.residue_hits += (uint32_t)H[3];
        info.window_hits += (uint32_t)H[4];
        info.hard_values += (uint32_t)H[5];
        info.update_bytes += (int64_t)(((uint64_t)(uint32_t)H[9] << 32) | (uint32_t)H[8]);
        info.filter_bytes += (int64_t)(((uint64_t)(uint32_t)H[11] << 32) | (uint32_t)H[10]);
        const int32_t* snapped = const_cast<const int32_t*>(H) + kModelHdr + 2 * n + (size_t)B * m->DWg + B;
        for (int j = 0; j < n; ++j) {
            ct_table_batch_done(b->tabs[j], H[kModelHdr + 2 * j], H[kModelHdr + 2 * j + 1], snapped[j] != 0);
            restPos[j] = -1;
        }
        nrest = 0;
        std::fill(dirty.begin(), dirty.end(), 0);
        const uint32_t* outDom = reinterpret_cast<const uint32_t*>(const_cast<const int32_t*>(b->h_status) + kModelHdr + 2 * n);
        const int32_t* outNode = const_cast<const int32_t*>(b->h_status) + kModelHdr + 2 * n + (size_t)B * m->DWg;
        (void)T;
        for (int s = 0; s < B; ++s)
            if (slots[s].pending)
                std::memcpy(slotDom(s), outDom + (size_t)s * m->DWg, (size_t)m->DWg * sizeof(uint32_t));
        scores = nullptr;
        if (usePolicy && !probeMode) {
            bool any = false;
            for (int s = 0; s < B; ++s) {
                b->h_active[s] = slots[s].pending && outNode[s] == CT_OK;
                any |= b->h_active[s] != 0;
            }
            if (any) {
                CT_CUDA(cudaMemcpyAsync(b->d_active, b->h_active.data(), (size_t)B, cudaMemcpyHostToDevice, b->stream));
                if ((rc = ct_feat_compute(b->fview, b->d_tabs, b->md.dom, b->d_active, b->stream)) != CT_OK) return rc;
                if ((rc = ct_feat_scores(b->fview, m->policy, b->stream)) != CT_OK) return rc;
                scores = b->fview->h_scores;
            }
        }
        for (int s = 0; s < B; ++s) {
            if (!slots[s].pending) continue;
            if (splitMode) {
                SplitOut& o = splitOut[s];
                o.status = outNode[s];
                o.x = o.status == CT_OK ? pick(s) : -1;
                o.dom.assign(slotDom(s), slotDom(s) + m->DWg);
                slots[s].pending = false;
                if ((rc = cancel(s)) != CT_OK) return rc;
                continue;
            }
            if (probeMode) {
                slots[s].pending = false;
                double L2 = 0.0;
                const uint32_t* dom = slotDom(s);
                for (int v = 0; v < m->nvars; ++v) L2 += std::log2((double)popcount_words(dom + m->off[v], m->nw[v]));
                probeLabel[s] = outNode[s] != CT_OK ? 1.0f : (float)((probeL - L2) / probeL);
                if ((rc = cancel(s)) != CT_OK) return rc;
                continue;
            }
            if ((rc = advance(s, outNode[s])) != CT_OK) return rc;
        }
        return CT_OK;
    }

    // ---- the slots' search on the device (count_all, first-fail) ----
    // The open nodes go to a device queue; the fixpoint kernel in search mode
    // decides for every slot between its rounds, launched again until the
    // search is done (each launch is bounded to kDevRoundBudget rounds).
    int run_device() {
        int rc;
        int L1 = 0;
        if ((rc = ct_model_save(m, &L1)) != CT_OK) return rc;
        rc = ct_model_propagate(m);  // the root fixpoint, for the state copies
        int levels = b && b->dsearch ? b->dsearch->maxLevels : kDevLevels;
        int factor = b && b->dsearch ? b->dsearch->trailFactor : kDevTrailFactor;
        for (;;) {
            if (rc == CT_OK) rc = ensure_copies();
            if (rc == CT_OK && b->dsearch && (b->dsearch->maxLevels < levels || b->dsearch->trailFactor < factor)) {
                dsearch_free(b->dsearch);
                b->dsearch = nullptr;
            }
            if (rc == CT_OK) rc = run_device_inner(levels, factor);
            // a subtree deeper, or a trail fuller, than the capacities: larger
            // ones, from the start again (the counts are the same)
            if (rc == CT_ERR_LEVEL && levels < kDevLevelsMax) {
                levels *= 2;
            } else if (rc == CT_ERR_OOM && devTrailFull && factor < kDevTrailFactorMax) {
                factor *= 2;
            } else {
                break;
            }
            b->broken = false;
            devRetries += 1;
            rc = CT_OK;
        }
        const int rr = ct_model_restore(m, L1);
        return rc != CT_OK ? rc : rr;
    }

    bool devTrailFull = false;
    int devRetries = 0;

    int run_device_inner(int levels, int factor) {
        int rc;
        devTrailFull = false;
        if (!b->dsearch) {
            DevSearch* nd = nullptr;
            rc = build_dsearch(m, b, levels, factor, &nd);
            if (rc != CT_OK) {
                dsearch_free(nd);
                return rc;
            }
            b->dsearch = nd;
        }
        DevSearch* d = b->dsearch;
        SearchDev S = d->hs;
        const int nopen = (int)open.size();
        const int DWs = m->DWg;
        if (nopen > d->nopenCap) {
            if (d->d_openDom) cudaFree(d->d_openDom);
            if (d->d_openDepth) cudaFree(d->d_openDepth);
            d->d_openDom = nullptr;
            d->d_openDepth = nullptr;
            d->nopenCap = 0;
            if (cudaMalloc(&d->d_openDom, (size_t)nopen * DWs * 4) != cudaSuccess ||
                cudaMalloc(&d->d_openDepth, (size_t)nopen * 4) != cudaSuccess) {
                cudaGetLastError();
                ct_set_error("device search: open-node queue of %d nodes", nopen);
                return CT_ERR_OOM;
            }
            d->nopenCap = nopen;
        }
        std::vector<uint32_t> od((size_t)nopen * DWs);
        std::vector<int32_t> odep(nopen);
        for (int o = 0; o < nopen; ++o) {
            std::memcpy(od.data() + (size_t)o * DWs, open[o].dom.data(), (size_t)DWs * 4);
            odep[o] = open[o].depth;
        }
        cudaStream_t str = b->stream;
        CT_CUDA(cudaMemcpyAsync(d->d_openDom, od.data(), od.size() * 4, cudaMemcpyHostToDevice, str));
        CT_CUDA(cudaMemcpyAsync(d->d_openDepth, odep.data(), odep.size() * 4, cudaMemcpyHostToDevice, str));
        CT_CUDA(cudaMemcpyAsync(d->d_root, rootDom.data(), (size_t)DWs * 4, cudaMemcpyHostToDevice, str));
        S.openDom = d->d_openDom;
        S.openDepth = d->d_openDepth;
        S.nopen = nopen;
        const int64_t remaining = limit > 0 ? std::max<int64_t>(limit - st.nodes, 0) : 0;
        S.nodeLimit = limit > 0 ? std::max<int64_t>(remaining, 0) : 0;
        if (limit > 0 && remaining == 0) {
            hitLimit = true;
            return CT_OK;
        }
        CT_CUDA(cudaMemcpyAsync(d->d_sd, &S, sizeof(S), cudaMemcpyHostToDevice, str));
        CT_CUDA(cudaMemsetAsync(S.ctr, 0, sizeof(SearchCtr), str));
        ModelDev md = b->md;
        CT_CUDA(cudaMemsetAsync(md.ctrl, 0, sizeof(ModelCtrl), str));
        md.tabs = d->d_tabs;
        md.search = d->d_sd;
        md.nrestores = 0;
        md.nworkIn = nullptr;
        CT_CUDA(launch_search_init(md, b->d_tabs, S, d->d_root, d->trailFactor, str));
        if (b->d_phase) CT_CUDA(cudaMemsetAsync(b->d_phase, 0, kModelPhases * sizeof(uint64_t), str));
        // the fixpoint launch's grid rule with the search variant's residency
        const int maxCoS = max_coresident_search_blocks();
        if (maxCoS <= 0) {
            ct_set_error("device search: the search kernel cannot be made resident on this device");
            return CT_ERR_CUDA;
        }
        const int searchGrid = m->opt.grid_blocks > 0 ? std::min(m->opt.grid_blocks, maxCoS) : maxCoS;
        SearchCtr c{};
        unsigned long long lastNodes = ~0ull;
        int idleLaunches = 0;
        volatile int32_t* H = b->h_status;
        for (;;) {
            H[0] = kNoChunk;
            const auto w0 = std::chrono::steady_clock::now();
            CT_CUDA(launch_model_search(md, searchGrid, str));
            bool seen = false;
            for (uint64_t it = 0;; ++it) {
                if (H[0] != kNoChunk) {
                    seen = true;
                    break;
                }
                if ((it & 1023u) == 1023u) {
                    if (cudaStreamQuery(str) == cudaSuccess) {
                        seen = H[0] != kNoChunk;
                        break;
                    }
                    if (std::chrono::steady_clock::now() - w0 > std::chrono::milliseconds(kHostWaitMs)) break;
                }
            }
            if (!seen) CT_CUDA(cudaStreamSynchronize(str));
            info.wait_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - w0).count();
            info.steps += 1;
            const int status = H[0];
            if (status != CT_OK) {
                b->broken = true;
                if (status == kNoChunk) {
                    ct_set_error("device search: the fixpoint kernel did not publish (a device-side wait ran out)");
                    return CT_ERR_TIMEOUT;
                }
                ct_set_error("device search: fixpoint kernel status %d (a trail overflow is CT_ERR_OOM)", status);
                devTrailFull = status == CT_ERR_OOM;
                return status < 0 ? status : CT_ERR_STATE;
            }
            st.propagations += H[2];
            info.rounds += H[1];
            CT_CUDA(cudaMemcpyAsync(&c, S.ctr, sizeof(c), cudaMemcpyDeviceToHost, str));
            CT_CUDA(cudaStreamSynchronize(str));
            if (c.done || c.error != CT_OK) break;
            // every launch issues nodes unless the search is stuck
            idleLaunches = c.nodes == lastNodes ? idleLaunches + 1 : 0;
            lastNodes = c.nodes;
            if (idleLaunches >= 2) {
                b->broken = true;
                ct_set_error("device search: no node issued in two launches");
                return CT_ERR_STATE;
            }
        }
        if (c.error != CT_OK) {
            ct_set_error("device search: %s", c.error == CT_ERR_LEVEL ? "a subtree is deeper than the device levels"
                                                                     : "stopped");
            return c.error;
        }
        if (b->d_phase) {
            // the phase clock (ct_options.profile): the rounds of the device search
            uint64_t ns[kModelPhases];
            CT_CUDA(cudaMemcpyAsync(ns, b->d_phase, sizeof(ns), cudaMemcpyDeviceToHost, str));
            CT_CUDA(cudaStreamSynchronize(str));
            for (int q = 0; q < kModelPhases; ++q) info.phase_seconds[q] = 1e-9 * (double)ns[q];
        }
        const int64_t issued = S.nodeLimit > 0 ? std::min<int64_t>((int64_t)c.nodes, S.nodeLimit) : (int64_t)c.nodes;
        if (S.nodeLimit > 0 && (int64_t)c.nodes >= S.nodeLimit) hitLimit = true;
        st.nodes += issued;
        st.fails += (int64_t)c.fails;
        st.solutions += (int64_t)c.solutions;
        st.max_depth = std::max(st.max_depth, c.maxDepth);
        info.slot_nodes += issued;
        info.open_nodes += std::min(c.nextOpen, nopen);
        if (c.solutions > 0) {
            // the first solution in depth-first order: the slots' first
            // solutions in their lowest open node, against the split's
            std::vector<int32_t> fo(B);
            CT_CUDA(cudaMemcpyAsync(fo.data(), S.firstOpen, (size_t)B * 4, cudaMemcpyDeviceToHost, str));
            CT_CUDA(cudaStreamSynchronize(str));
            int bs = -1;
            for (int q = 0; q < B; ++q)
                if (fo[q] < nopen && (bs < 0 || fo[q] < fo[bs])) bs = q;
            if (bs >= 0 && (!haveBest || after(bestPath, open[fo[bs]].path))) {
                std::vector<uint32_t> sol(DWs);
                CT_CUDA(cudaMemcpyAsync(sol.data(), S.firstSol + (size_t)bs * DWs, (size_t)DWs * 4,
                                        cudaMemcpyDeviceToHost, str));
                CT_CUDA(cudaStreamSynchronize(str));
                haveBest = true;
                bestPath = open[fo[bs]].path;
                bestVals.resize(m->nvars);
                for (int v = 0; v < m->nvars; ++v) bestVals[v] = m->lo[v] + min_value(m, sol.data(), v);
            }
        }
        return CT_OK;
    }

    int run_slots() {
        // a named range for profilers (no cost without one attached)
        nvtxRangePushA("ct_search_batch_slots");
        const int rc = run_slots_timed();
        nvtxRangePop();
        return rc;
    }

    int run_slots_timed() {
        const auto s0 = std::chrono::steady_clock::now();
        if (b->d_phase) CT_CUDA(cudaMemsetAsync(b->d_phase, 0, kModelPhases * sizeof(uint64_t), b->stream));
        int rc = run_slots_inner();
        if (rc == CT_OK && b->d_phase) {
            uint64_t ns[kModelPhases];
            CT_CUDA(cudaMemcpyAsync(ns, b->d_phase, sizeof(ns), cudaMemcpyDeviceToHost, b->stream));
            CT_CUDA(cudaStreamSynchronize(b->stream));
            for (int p = 0; p < kModelPhases; ++p) info.phase_seconds[p] = 1e-9 * (double)ns[p];
        }
        info.slot_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - s0).count();
        return rc;
    }

    // Idle slots at the root state (kept when the split phase already ran in
    // them: their undos may still be staged for the next launch).
    void init_slots() {
        if (slotsReady) return;
        const int n = b->n;
        slots.assign(B, Slot());
        dirty.assign(n, 0);
        restPos.assign(n, -1);
        nrest = 0;
        for (int s = 0; s < B; ++s) std::memcpy(slotDom(s), rootDom.data(), (size_t)m->DWg * sizeof(uint32_t));
        slotsReady = true;
    }

    int run_slots_inner() {
        init_slots();
        for (;;) {
            for (int s = 0; s < B; ++s) {
                if (slots[s].active) continue;
                const int rc = assign(s);
                if (rc != CT_OK) return rc;
            }
            bool any = nrest > 0;
            for (int s = 0; s < B && !any; ++s) any = slots[s].pending;
            if (!any) break;
            const int rc = step();
            if (rc != CT_OK) return rc;
        }
        return CT_OK;
    }
};

}  // namespace

namespace {
int search_batch(ct_model* m, int slots, int split_depth, bool split_assign, int64_t node_limit, int count_all,
                 ct_search_stats* out, int32_t* first_solution, ct_batch_info* info, bool on_device = false);
}  // namespace

extern "C" int ct_search_batch_device(ct_model* m, int slots, int split_depth, int64_t node_limit,
                                      ct_search_stats* out, int32_t* first_solution, ct_batch_info* info) {
    if (m && m->policy) {
        ct_set_error("ct_search_batch_device: branches first-fail only (the model has a policy set)");
        return CT_ERR_ARG;
    }
    return search_batch(m, slots, split_depth, false, node_limit, 1, out, first_solution, info, true);
}

extern "C" int ct_search_batch(ct_model* m, int slots, int split_depth, int64_t node_limit, int count_all,
                               ct_search_stats* out, int32_t* first_solution, ct_batch_info* info) {
    return search_batch(m, slots, split_depth, false, node_limit, count_all, out, first_solution, info);
}

extern "C" int ct_search_batch_assign(ct_model* m, int slots, int assign_depth, int64_t node_limit, int count_all,
                                      ct_search_stats* out, int32_t* first_solution, ct_batch_info* info) {
    if (assign_depth < 1 || assign_depth > 16 || count_all == 2) {
        ct_set_error("ct_search_batch_assign: assign_depth %d out of [1, 16] or count_all %d", assign_depth, count_all);
        return CT_ERR_ARG;
    }
    return search_batch(m, slots, assign_depth, true, node_limit, count_all, out, first_solution, info);
}

namespace {
int search_batch(ct_model* m, int slots, int split_depth, bool split_assign, int64_t node_limit, int count_all,
                 ct_search_stats* out, int32_t* first_solution, ct_batch_info* info, bool on_device) {
    if (!m || !out) {
        ct_set_error("ct_search_batch: null argument");
        return CT_ERR_ARG;
    }
    if (slots < 1 || slots > 4096 || split_depth < 0 || split_depth > 64 || count_all < 0 || count_all > 2 ||
        (int64_t)slots * (int64_t)m->tables.size() > kModelMaxTables) {
        ct_set_error("ct_search_batch: slots %d or split depth %d out of range", slots, split_depth);
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_search_batch: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    if (info) std::memset(info, 0, sizeof(*info));
    if (m->tables.empty() || m->staticInfeasible) {
        // nothing to propagate on the device: the plain search is the same search
        const int rc = ct_search_dfs(m, node_limit, count_all == 1, out, first_solution);
        if (info) {
            info->slots = slots;
            info->split_nodes = rc == CT_OK ? out->nodes : 0;
        }
        return rc;
    }
    Search S;
    S.t0 = std::chrono::steady_clock::now();
    S.m = m;
    S.b = m->bsearch;
    S.B = slots;
    S.splitDepth = split_depth;
    S.splitAssign = split_assign;
    S.limit = node_limit;
    S.countAll = count_all == 1;
    S.anyStop = count_all == 2;
    // the device search keeps no slot waiting for another's right branches:
    // it splits on until every slot has several open nodes to take
    if (on_device) S.minOpen = (int64_t)kDevOpenPerSlot * slots;
    // any solution: the model first searches alone for 4 nodes per slot; easy
    // instances end there, the others continue from the frontier it leaves
    if (S.anyStop) S.splitBudget = 4 * (int64_t)slots;
    S.usePolicy = m->policy != nullptr;
    const int64_t p0 = m->propagations;
    int L0 = 0;
    int rc = ct_model_save(m, &L0);
    if (rc != CT_OK) return rc;
    std::vector<uint8_t> path;
    // the breadth-first split in the slots, except for the budgeted
    // any-solution search (the model searches its share depth-first first)
    if ((split_depth >= 2 || split_assign || on_device) && !S.anyStop) {
        rc = S.split_bfs();
    } else {
        if (split_depth == 0) rc = S.ensure_copies();
        if (rc == CT_OK) rc = S.split(0, path);
    }
    const int rr = ct_model_restore(m, L0);
    if (rc == CT_OK) rc = rr;
    const bool runSlots = !S.open.empty() && !S.stopIssue && !(S.anyStop && S.haveBest);
    if (rc == CT_OK && runSlots && S.usePolicy) rc = ensure_slot_features(m, S.b);
    if (rc == CT_OK && runSlots) rc = on_device ? S.run_device() : S.run_slots();
    if (rc != CT_OK) {
        if (S.b) S.b->broken = true;
        return rc;
    }
    CT_CUDA(cudaStreamSynchronize(m->stream));
    S.st.propagations += m->propagations - p0;
    S.st.complete = S.hitLimit ? 0 : 1;
    S.st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
    *out = S.st;
    if (first_solution && S.haveBest) std::memcpy(first_solution, S.bestVals.data(), S.bestVals.size() * sizeof(int32_t));
    if (info) {
        *info = S.info;
        info->slots = slots;
        info->split_depth = split_depth;
    }
    return CT_OK;
}
}  // namespace

extern "C" int ct_model_lookahead(ct_model* m, int slots, float* labels_host) {
    if (!m || !labels_host || slots < 1 || slots > 4096 || (int64_t)slots * (int64_t)m->tables.size() > kModelMaxTables) {
        ct_set_error("ct_model_lookahead: bad argument");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_model_lookahead: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    if (m->hasNegative) {
        ct_set_error("ct_model_lookahead: not available for models with negative tables");
        return CT_ERR_ARG;
    }
    int rc = ct_model_propagate(m);
    if (rc != CT_OK) return rc;
    std::vector<int> cand;
    double L = 0.0;
    for (int v = 0; v < m->nvars; ++v) {
        const int sz = ct_model_popcount_var(m, v);
        labels_host[v] = std::nanf("");
        L += std::log2((double)sz);
        if (sz > 1) cand.push_back(v);
    }
    if (cand.empty()) return CT_OK;
    if (m->tables.empty()) {
        // no constraint: fixing x removes log2|D(x)| and nothing else
        for (int v : cand) labels_host[v] = (float)(std::log2((double)ct_model_popcount_var(m, v)) / L);
        return CT_OK;
    }
    Search S;
    S.m = m;
    S.b = m->bsearch;
    S.B = slots;
    S.probeMode = true;
    S.probeL = L;
    if ((rc = S.ensure_copies()) != CT_OK) return rc;
    const int n = S.b->n;
    S.slots.assign(slots, Slot());
    S.dirty.assign(n, 0);
    S.restPos.assign(n, -1);
    S.probeLabel.assign(slots, 0.0f);
    for (int s = 0; s < slots; ++s) std::memcpy(S.slotDom(s), S.rootDom.data(), (size_t)m->DWg * sizeof(uint32_t));
    std::vector<uint32_t> probe;
    for (size_t c0 = 0; c0 < cand.size(); c0 += (size_t)slots) {
        const int cnt = (int)std::min<size_t>((size_t)slots, cand.size() - c0);
        for (int s = 0; s < cnt; ++s) {
            const int x = cand[c0 + s];
            probe = S.rootDom;
            const int a = min_value(m, probe.data(), x);
            for (int q = 0; q < m->nw[x]; ++q) probe[m->off[x] + q] = 0u;
            probe[m->off[x] + (a >> 5)] = 1u << (a & 31);
            Slot& Z = S.slots[s];
            if ((rc = S.save_slot(s)) != CT_OK) return rc;
            std::memcpy(S.slotDom(s), probe.data(), (size_t)m->DWg * sizeof(uint32_t));
            for (int k = 0; k < S.b->T; ++k) S.dirty[(size_t)s * S.b->T + k] = 1;
            Z.active = true;
            Z.pending = true;
        }
        if ((rc = S.step()) != CT_OK) return rc;
        for (int s = 0; s < cnt; ++s) labels_host[cand[c0 + s]] = S.probeLabel[s];
    }
    return CT_OK;
}

namespace {

struct Collect {
    int slots;
    int64_t max;
    float* X;
    float* y;
    int64_t n = 0;
    std::vector<float> feat, lab;
};

int collect_hook(void* ctx, ct_model* m) {
    Collect* c = static_cast<Collect*>(ctx);
    if (c->n >= c->max) return CT_OK;
    c->feat.resize((size_t)m->nvars * kNF);
    c->lab.resize((size_t)m->nvars);
    int rc = ct_model_features(m, c->feat.data());
    if (rc == CT_OK) rc = ct_model_lookahead(m, c->slots, c->lab.data());
    if (rc != CT_OK) return rc;
    for (int v = 0; v < m->nvars && c->n < c->max; ++v) {
        if (ct_model_popcount_var(m, v) < 2) continue;
        std::memcpy(c->X + (size_t)c->n * kNF, c->feat.data() + (size_t)v * kNF, kNF * sizeof(float));
        c->y[c->n] = c->lab[v];
        ++c->n;
    }
    return CT_OK;
}

}  // namespace

extern "C" int ct_search_collect(ct_model* m, int64_t node_limit, int slots, int64_t max_samples, float* features_host,
                                 float* labels_host, int64_t* samples_out) {
    if (!m || !features_host || !labels_host || !samples_out || max_samples < 0 || slots < 1 || slots > 4096) {
        ct_set_error("ct_search_collect: bad argument");
        return CT_ERR_ARG;
    }
    Collect c;
    c.slots = slots;
    c.max = max_samples;
    c.X = features_host;
    c.y = labels_host;
    ct_search_stats st{};
    const int rc = ct_model_dfs(m, node_limit, true, false, &st, nullptr, collect_hook, &c);
    *samples_out = c.n;
    return rc;
}

