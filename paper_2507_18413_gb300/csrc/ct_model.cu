// ct_model.cu -- networks of table constraints: propagation to a common
// fixpoint and depth-first search (Sec. 4: the solver alternates search and
// propagation, backtracking through the trail; Sec. 2: propagation removes
// unsupported values until GAC holds or a failure is found).
//
// All domains live in one device array; every table reads and prunes its
// scope variables in place. By default the whole fixpoint is one cooperative
// launch (ct_model_kernel): rounds of all dirty tables propagated together,
// removals applied together, until no table needs another pass. With
// ct_options.host_fixpoint the queue runs on the host instead: after each
// table propagation the host learns which scope variables changed and
// schedules the other tables that share them. Either way one table pass is
// GAC for that table, so a table is not re-queued by its own pruning.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include "ct_model.cuh"

using namespace ctk;

namespace {

template <typename T>
int m_alloc(ct_model* m, T** p, size_t n) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("model: cudaMalloc: %s", cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return CT_OK;
}

// The device domains made equal to the host copy when a set or a restore
// changed the host copy since the last upload (synchronous: the staging
// buffer is free again on return).
int sync_dom(ct_model* m) {
    if (!m->domStale) return CT_OK;
    std::memcpy(m->h_stage, m->h_dom.data(), (size_t)m->DWg * sizeof(uint32_t));
    CT_CUDA(cudaMemcpyAsync(m->d_dom, m->h_stage, (size_t)m->DWg * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    m->domStale = false;
    return CT_OK;
}

// Device descriptors of the network for the one-launch fixpoint (built once,
// after the last table was added).
int batch_setup(ct_model* m) {
    const int n = (int)m->tables.size();
    std::vector<int32_t> base(n + 1, 0), off, var;
    for (int t = 0; t < n; ++t) {
        base[t + 1] = base[t] + (int)m->scopes[t].size();
        for (int k = 0; k < (int)m->scopes[t].size(); ++k) {
            off.push_back(m->tabOff[t][k]);
            var.push_back(m->scopes[t][k]);
        }
    }
    ModelDev& M = m->md;
    int st;
    int32_t *dBase, *dOff, *dVar, *dPruned, *dNode;
    ModelCtrl* dCtrl;
    if ((st = m_alloc(m, &m->d_tabs, n)) != CT_OK) return st;
    // One block, its head copied at once per launch: [count, 3 pad | calls[n] |
    // domains[DWg] | work[2][n]]; the domains move into it.
    const size_t blkWords = 4 + 4 * (size_t)n + (size_t)m->DWg + 2 * (size_t)n;
    static_assert(sizeof(ModelTabCall) == 4 * sizeof(int32_t), "ModelTabCall is four words");
    if ((st = m_alloc(m, &m->d_blk, blkWords)) != CT_OK) return st;
    m->d_calls = reinterpret_cast<ModelTabCall*>(m->d_blk + 4);
    uint32_t* blkDom = reinterpret_cast<uint32_t*>(m->d_blk + 4 + 4 * (size_t)n);
    if ((st = sync_dom(m)) != CT_OK) return st;
    CT_CUDA(cudaMemcpyAsync(blkDom, m->d_dom, (size_t)m->DWg * sizeof(uint32_t), cudaMemcpyDeviceToDevice, m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    cudaFree(m->d_dom);
    m->d_dom = blkDom;
    m->domInBlk = true;
    if ((st = m_alloc(m, &dBase, n + 1)) != CT_OK) return st;
    if ((st = m_alloc(m, &dOff, off.size())) != CT_OK) return st;
    if ((st = m_alloc(m, &dVar, var.size())) != CT_OK) return st;
    M.work = m->d_blk + 4 + 4 * (size_t)n + m->DWg;
    if ((st = m_alloc(m, &M.unitPrefix, (size_t)n + 1)) != CT_OK) return st;
    if ((st = m_alloc(m, &M.rowPrefix, (size_t)n + 1)) != CT_OK) return st;
    if ((st = m_alloc(m, &dPruned, 2 * (size_t)m->nvars)) != CT_OK) return st;
    if ((st = m_alloc(m, &M.snapTaken, (size_t)n)) != CT_OK) return st;
    CT_CUDA(cudaMemsetAsync(M.snapTaken, 0, std::max<size_t>(n, 1) * sizeof(int32_t), m->stream));
    if ((st = m_alloc(m, &dCtrl, 1)) != CT_OK) return st;
    const int nodeTables = std::max(n, 1);  // the whole network is one node
    const int nnodes = 1;
    if ((st = m_alloc(m, &dNode, (size_t)nnodes)) != CT_OK) return st;
    CT_CUDA(cudaMemsetAsync(dNode, 0, (size_t)nnodes * sizeof(int32_t), m->stream));
    CT_CUDA(cudaMemcpyAsync(dBase, base.data(), base.size() * 4, cudaMemcpyHostToDevice, m->stream));
    if (!off.empty()) {
        CT_CUDA(cudaMemcpyAsync(dOff, off.data(), off.size() * 4, cudaMemcpyHostToDevice, m->stream));
        CT_CUDA(cudaMemcpyAsync(dVar, var.data(), var.size() * 4, cudaMemcpyHostToDevice, m->stream));
    }
    CT_CUDA(cudaMemsetAsync(dPruned, 0xff, 2 * (size_t)m->nvars * 4, m->stream));
    CT_CUDA(cudaMemsetAsync(dCtrl, 0, sizeof(ModelCtrl), m->stream));
    if (cudaHostAlloc((void**)&m->h_blk, blkWords * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&m->h_mstatus, (size_t)(kModelHdr + 2 * n + m->DWg + nnodes + n) * sizeof(int32_t),
                      cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("model: pinned host buffers");
        return CT_ERR_OOM;
    }
    int32_t* dStatus = nullptr;
    CT_CUDA(cudaHostGetDevicePointer((void**)&dStatus, m->h_mstatus, 0));
    m->h_calls = reinterpret_cast<ModelTabCall*>(m->h_blk + 4);
    m->h_list = m->h_blk + 4 + 4 * (size_t)n + m->DWg;
    M.tabs = m->d_tabs;
    M.calls = m->d_calls;
    M.nworkIn = m->d_blk;
    M.scopeBase = dBase;
    M.scopeOff = dOff;
    M.scopeVar = dVar;
    M.prunedBy = dPruned;
    M.nodeStatus = dNode;
    M.nodeTables = nodeTables;
    M.ctrl = dCtrl;
    M.dom = m->d_dom;
    M.statusBlk = dStatus;
    M.ntables = n;
    M.nvars = m->nvars;
    M.DWg = m->DWg;
    int64_t domBits = 0;
    for (int v = 0; v < m->nvars; ++v) domBits += m->size[v];
    M.maxRounds = (int)std::min<int64_t>(domBits + 2, 1 << 30);
    m->tabVersion.assign(n, -1);
    const int maxCo = max_coresident_model_blocks(n);
    if (maxCo <= 0) {
        ct_set_error("model: the fixpoint kernel cannot be made resident on this device");
        return CT_ERR_CUDA;
    }
    int64_t segs = 0, rows = 0;
    for (ct_table* tab : m->tables) {
        segs += ct_table_dev(tab).nseg;
        rows += ct_table_dev(tab).R;
    }
    if ((st = m_alloc(m, &M.missQ, (size_t)std::max<int64_t>(rows, 1))) != CT_OK) return st;
    if (m->opt.profile) {
        if ((st = m_alloc(m, &M.phaseNs, kModelPhases)) != CT_OK) return st;
        CT_CUDA(cudaMemsetAsync(M.phaseNs, 0, kModelPhases * sizeof(uint64_t), m->stream));
    }
    int64_t want = std::max<int64_t>({(int64_t)n, (segs + kWarps - 1) / kWarps, (rows + 2 * kWarps - 1) / (2 * kWarps), 1});
    if (m->opt.grid_blocks > 0) want = m->opt.grid_blocks;
    m->grid = (int)std::min<int64_t>(want, maxCo);
    CT_CUDA(cudaStreamSynchronize(m->stream));
    m->batchReady = true;
    return CT_OK;
}

int batch_propagate(ct_model* m);
int popcount_var(const ct_model* m, int v);
int set_var(ct_model* m, int v, const uint32_t* words);

// CTA count of the fixpoint launch chosen by trial fixpoints (ct_options.autotune):
// half of the 4 largest domains removed, propagated, restored; best of 3 per candidate.
int tune_grid(ct_model* m) {
    const int maxCo = max_coresident_model_blocks((int)m->tables.size());
    if (maxCo <= 0 || m->tables.empty()) return CT_OK;
    const int want = m->grid;
    std::vector<int> cands;
    for (int g : {want / 4, want / 2, want, 2 * want, maxCo / 2, maxCo}) {
        g = std::max(1, std::min(g, maxCo));
        if (std::find(cands.begin(), cands.end(), g) == cands.end()) cands.push_back(g);
    }
    std::vector<int> order(m->nvars);
    for (int v = 0; v < m->nvars; ++v) order[v] = v;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return popcount_var(m, a) > popcount_var(m, b); });
    double best = 1e30;
    int bestGrid = want;
    int st = CT_OK;
    for (int g : cands) {
        m->grid = g;
        double tmin = 1e30;
        for (int rep = 0; rep < 3 && st == CT_OK; ++rep) {
            int L = 0;
            if ((st = ct_model_save(m, &L)) != CT_OK) break;
            for (int k = 0; k < std::min(4, m->nvars); ++k) {
                const int v = order[k];
                std::vector<uint32_t> w(m->h_dom.begin() + m->off[v], m->h_dom.begin() + m->off[v] + m->nw[v]);
                int seen = 0, keep = std::max(1, popcount_var(m, v) / 2);
                for (int q = 0; q < m->nw[v]; ++q)
                    for (int b = 0; b < 32; ++b)
                        if ((w[q] >> b) & 1u) {
                            if (seen >= keep) w[q] &= ~(1u << b);
                            ++seen;
                        }
                if ((st = set_var(m, v, w.data())) != CT_OK) break;
            }
            const auto t0 = std::chrono::steady_clock::now();
            const int r = st == CT_OK ? batch_propagate(m) : st;
            tmin = std::min(tmin, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
            if (r < 0) st = r;
            const int rr = ct_model_restore(m, L);
            if (st == CT_OK) st = rr;
        }
        if (st != CT_OK) break;
        if (tmin < best) {
            best = tmin;
            bestGrid = g;
        }
    }
    m->grid = st == CT_OK ? bestGrid : want;
    m->stats = ct_model_stats{};
    m->propagations = 0;
    return st;
}

int batch_propagate(ct_model* m) {
    int st;
    if (!m->batchReady) {
        if ((st = batch_setup(m)) != CT_OK) return st;
        if (m->opt.autotune && m->opt.grid_blocks <= 0 && (st = tune_grid(m)) != CT_OK) return st;
    }
    const int n = (int)m->tables.size();
    int nwork = 0;
    for (int t = 0; t < n; ++t) {
        if ((st = ct_table_batch_prepare(m->tables[t], &m->h_calls[t])) != CT_OK) return st;
        if (m->dirty[t]) m->h_list[nwork++] = t;
    }
    if (nwork == 0) return CT_OK;
    // device copies of the tables whose buffers moved (trail or level growth)
    for (int t = 0; t < n; ++t) {
        const int v = ct_table_version(m->tables[t]);
        if (v != m->tabVersion[t]) {
            CT_CUDA(cudaMemcpyAsync(m->d_tabs + t, &ct_table_dev(m->tables[t]), sizeof(TableDev), cudaMemcpyHostToDevice,
                                    m->stream));
            m->tabVersion[t] = v;
        }
    }
    // count, calls, domains (the host copy is authoritative) and the first
    // round's tables in one copy
    m->h_blk[0] = nwork;
    std::memcpy(m->h_blk + 4 + 4 * (size_t)n, m->h_dom.data(), (size_t)m->DWg * sizeof(uint32_t));
    CT_CUDA(cudaMemcpyAsync(m->d_blk, m->h_blk, (4 + 4 * (size_t)n + (size_t)m->DWg + (size_t)nwork) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, m->stream));
    m->domStale = false;
    volatile int32_t* H = m->h_mstatus;
    H[0] = kNoChunk;
    const auto t0 = std::chrono::steady_clock::now();
    CT_CUDA(launch_model(m->md, m->grid, m->stream));
    bool seen = false;
    for (uint64_t it = 0;; ++it) {
        if (H[0] != kNoChunk) {
            seen = true;
            break;
        }
        if ((it & 1023u) == 1023u && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(kHostWaitMs))
            break;
    }
    if (!seen) CT_CUDA(cudaStreamSynchronize(m->stream));
    m->stats.wait_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const int status = H[0];
    if (status == kNoChunk) {
        ct_set_error("model: the fixpoint kernel did not publish (a device-side wait ran out)");
        m->batch = false;
        m->failed = true;
        return CT_ERR_TIMEOUT;
    }
    m->propagations += H[2];
    m->stats.fixpoints += 1;
    m->stats.rounds += H[1];
    m->stats.propagations += H[2];
    m->stats.residue_hits += (uint32_t)H[3];
    m->stats.window_hits += (uint32_t)H[4];
    m->stats.hard_values += (uint32_t)H[5];
    m->stats.update_bytes += (int64_t)(((uint64_t)(uint32_t)H[9] << 32) | (uint32_t)H[8]);
    m->stats.filter_bytes += (int64_t)(((uint64_t)(uint32_t)H[11] << 32) | (uint32_t)H[10]);
    const int32_t* snapped = const_cast<const int32_t*>(H) + kModelHdr + 2 * n + m->DWg + 1;  // after the one node
    for (int t = 0; t < n; ++t)
        ct_table_batch_done(m->tables[t], H[kModelHdr + 2 * t], H[kModelHdr + 2 * t + 1], snapped[t] != 0);
    if (status == CT_OK && H[kModelHdr + 2 * n + m->DWg] == CT_INFEASIBLE) {
        m->failed = true;
        return CT_INFEASIBLE;
    }
    if (status != CT_OK) {
        m->failed = true;
        ct_set_error("model: fixpoint kernel status %d", status);
        return status;
    }
    const uint32_t* outDom = reinterpret_cast<const uint32_t*>(const_cast<const int32_t*>(m->h_mstatus) + kModelHdr + 2 * n);
    std::memcpy(m->h_dom.data(), outDom, (size_t)m->DWg * sizeof(uint32_t));
    std::fill(m->dirty.begin(), m->dirty.end(), 0);
    return CT_OK;
}

int popcount_var(const ct_model* m, int v) {
    int s = 0;
    for (int q = 0; q < m->nw[v]; ++q) s += __builtin_popcount(m->h_dom[(size_t)m->off[v] + q]);
    return s;
}

void mark_var(ct_model* m, int v, int except, std::deque<int>* q) {
    for (int T : m->varTables[v]) {
        if (T == except || m->dirty[T]) continue;
        m->dirty[T] = 1;
        if (q) q->push_back(T);
    }
}

// Replace the domain of variable v, scheduling its tables. The host copy is
// authoritative; the device copy follows with the next fixpoint launch (or
// sync_dom).
int set_var(ct_model* m, int v, const uint32_t* words) {
    std::memcpy(m->h_dom.data() + m->off[v], words, (size_t)m->nw[v] * sizeof(uint32_t));
    m->domStale = true;
    mark_var(m, v, -1, nullptr);
    return CT_OK;
}

}  // namespace

int ct_model_popcount_var(const ct_model* m, int v) { return popcount_var(m, v); }

namespace {

// The model's feature view and an up-to-date device copy of every table.
int ensure_features(ct_model* m) {
    int st;
    if (m->hasNegative) {
        ct_set_error("features: not defined for models with negative tables");
        return CT_ERR_ARG;
    }
    if (!m->batchReady && (st = batch_setup(m)) != CT_OK) return st;
    const int n = (int)m->tables.size();
    for (int t = 0; t < n; ++t) {
        const int v = ct_table_version(m->tables[t]);
        if (v != m->tabVersion[t]) {
            CT_CUDA(cudaMemcpyAsync(m->d_tabs + t, &ct_table_dev(m->tables[t]), sizeof(TableDev), cudaMemcpyHostToDevice,
                                    m->stream));
            m->tabVersion[t] = v;
        }
    }
    if (m->fview) return CT_OK;
    std::vector<int> R(n), seg(n);
    for (int t = 0; t < n; ++t) {
        R[t] = ct_table_dev(m->tables[t]).R;
        seg[t] = ct_table_dev(m->tables[t]).nseg;
    }
    FeatView* f = new (std::nothrow) FeatView();
    if (!f) return CT_ERR_OOM;
    st = ct_feat_view_build(f, 1, m->scopes, R, seg, m->off, m->nw, m->size, m->DWg);
    if (st != CT_OK) {
        ct_feat_view_free(f);
        delete f;
        return st;
    }
    m->fview = f;
    return CT_OK;
}

}  // namespace

int ct_model_pick_var(ct_model* m, bool usePolicy, int* x) {
    *x = -1;
    const float* sc = nullptr;
    if (usePolicy && m->policy) {
        bool any = false;
        for (int v = 0; v < m->nvars && !any; ++v) any = popcount_var(m, v) > 1;
        if (!any) return CT_OK;
        int st = ensure_features(m);
        if (st == CT_OK) st = sync_dom(m);
        if (st == CT_OK) st = ct_feat_compute(m->fview, m->d_tabs, m->d_dom, nullptr, m->stream);
        if (st == CT_OK) st = ct_feat_scores(m->fview, m->policy, m->stream);
        if (st != CT_OK) return st;
        sc = m->fview->h_scores;
    }
    int best = 0;
    float bestScore = 0.0f;
    for (int v = 0; v < m->nvars; ++v) {
        const int s = popcount_var(m, v);
        if (s < 2) continue;
        if (sc) {
            if (*x < 0 || sc[v] > bestScore) {
                *x = v;
                bestScore = sc[v];
            }
        } else if (*x < 0 || s < best) {
            *x = v;
            best = s;
        }
    }
    return CT_OK;
}
int ct_model_set_var(ct_model* m, int v, const uint32_t* words) { return set_var(m, v, words); }

extern "C" int ct_model_create(int nvars, const int32_t* dom_lo, const int32_t* dom_size, const ct_options* opt,
                               void* cuda_stream, ct_model** out) {
    if (!out || nvars < 1 || !dom_lo || !dom_size) {
        ct_set_error("ct_model_create: bad argument");
        return CT_ERR_ARG;
    }
    *out = nullptr;
    for (int v = 0; v < nvars; ++v) {
        if (dom_size[v] < 1 || dom_size[v] > kMaxDomSize) {
            ct_set_error("ct_model_create: dom_size[%d] = %d out of range", v, dom_size[v]);
            return CT_ERR_ARG;
        }
    }
    ct_model* m = new (std::nothrow) ct_model();
    if (!m) return CT_ERR_OOM;
    m->nvars = nvars;
    m->lo.assign(dom_lo, dom_lo + nvars);
    m->size.assign(dom_size, dom_size + nvars);
    m->nw.resize(nvars);
    m->off.resize(nvars);
    for (int v = 0; v < nvars; ++v) {
        m->nw[v] = (m->size[v] + 31) / 32;
        m->off[v] = m->DWg;
        m->DWg += m->nw[v];
    }
    m->varTables.resize(nvars);
    m->h_dom.assign(m->DWg, 0u);
    for (int v = 0; v < nvars; ++v)
        for (int a = 0; a < m->size[v]; ++a) m->h_dom[(size_t)m->off[v] + a / 32] |= 1u << (a % 32);
    if (opt) m->opt = *opt;
    m->batch = !(opt && opt->host_fixpoint);
    cudaError_t e;
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete m;
            return ct_cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        m->ownStream = true;
    }
    e = cudaMalloc(&m->d_dom, (size_t)m->DWg * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&m->h_stage, (size_t)m->DWg * sizeof(uint32_t), cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_dom, m->h_dom.data(), (size_t)m->DWg * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        const int st = ct_cuda_fail(e, "model domain array");
        ct_model_destroy(m);
        return st;
    }
    *out = m;
    return CT_OK;
}

namespace {
int add_table_impl(ct_model* m, const int32_t* scope, int arity, const int32_t* tuples, int64_t t, bool negative);
}  // namespace

extern "C" int ct_model_add_table(ct_model* m, const int32_t* scope, int arity, const int32_t* tuples, int64_t t) {
    return add_table_impl(m, scope, arity, tuples, t, false);
}

extern "C" int ct_model_add_negative_table(ct_model* m, const int32_t* scope, int arity, const int32_t* tuples,
                                           int64_t t) {
    return add_table_impl(m, scope, arity, tuples, t, true);
}

namespace {
int add_table_impl(ct_model* m, const int32_t* scope, int arity, const int32_t* tuples, int64_t t, bool negative) {
    if (!m || !scope || arity < 1 || arity > kMaxArity) {
        ct_set_error("ct_model_add_table: bad argument");
        return CT_ERR_ARG;
    }
    if (!m->levels.empty() || m->batchReady) {
        ct_set_error("ct_model_add_table: tables must be added before the first save or propagation");
        return CT_ERR_STATE;
    }
    std::vector<int> sc(scope, scope + arity);
    std::vector<char> seen(m->nvars, 0);
    for (int v : sc) {
        if (v < 0 || v >= m->nvars || seen[v]) {
            ct_set_error("ct_model_add_table: scope variable %d out of range or repeated", v);
            return CT_ERR_ARG;
        }
        seen[v] = 1;
    }
    std::vector<int32_t> lo(arity), sz(arity), offs(arity);
    for (int k = 0; k < arity; ++k) {
        lo[k] = m->lo[sc[k]];
        sz[k] = m->size[sc[k]];
        offs[k] = m->off[sc[k]];
    }
    ct_table* tab = nullptr;
    const int st = negative ? ct_create_negative(arity, lo.data(), sz.data(), tuples, t, &m->opt, m->stream, &tab)
                            : ct_create(arity, lo.data(), sz.data(), tuples, t, &m->opt, m->stream, &tab);
    if (st < 0) return st;
    if (negative) m->hasNegative = true;  // no ordering features (they count positive supports)
    int32_t* d_off = nullptr;
    cudaError_t e = cudaMalloc(&d_off, (size_t)arity * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, offs.data(), (size_t)arity * sizeof(int32_t), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        if (d_off) cudaFree(d_off);
        ct_destroy(tab);
        return ct_cuda_fail(e, "ct_model_add_table offsets");
    }
    const int T = (int)m->tables.size();
    m->tables.push_back(tab);
    m->scopes.push_back(sc);
    m->d_tabOff.push_back(d_off);
    m->tabOff.push_back(offs);
    m->dirty.push_back(1);
    for (int v : sc) m->varTables[v].push_back(T);
    if (st == CT_INFEASIBLE) m->staticInfeasible = true;
    return st;
}
}  // namespace

extern "C" int ct_model_propagate(ct_model* m) {
    if (!m) {
        ct_set_error("ct_model_propagate: null handle");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_model_propagate: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    if (m->staticInfeasible) {
        m->failed = true;
        return CT_INFEASIBLE;
    }
    for (int v = 0; v < m->nvars; ++v) {
        if (popcount_var(m, v) == 0) {
            m->failed = true;
            return CT_INFEASIBLE;
        }
    }
    if (m->batch && (int)m->tables.size() <= kModelMaxTables) return batch_propagate(m);
    if (const int sst = sync_dom(m); sst != CT_OK) return sst;
    std::deque<int> q;
    for (int T = 0; T < (int)m->tables.size(); ++T)
        if (m->dirty[T]) q.push_back(T);
    std::vector<uint32_t> changed;
    while (!q.empty()) {
        const int T = q.front();
        q.pop_front();
        m->dirty[T] = 0;
        ct_table* tab = m->tables[T];
        changed.assign((size_t)ct_table_changed_words(tab), 0u);
        const int st = ct_table_propagate_on(tab, m->d_dom, m->d_tabOff[T], m->tabOff[T].data(), changed.data());
        m->propagations += 1;
        m->stats.propagations += 1;
        if (st == CT_INFEASIBLE) {
            m->failed = true;
            return CT_INFEASIBLE;
        }
        if (st < 0) return st;
        const int32_t* h = ct_table_status_host(tab);
        const uint32_t* newDom = reinterpret_cast<const uint32_t*>(h + kStatusHdr + ct_table_changed_words(tab));
        const int32_t* ld = ct_table_var_ld(tab);
        const std::vector<int>& sc = m->scopes[T];
        // One pass of a positive table is GAC for it; a negative table's pass is
        // not (a removal shrinks the other variables' products), so it is
        // scheduled again by its own removals.
        const int self = ct_table_is_negative(tab) ? -1 : T;
        for (int k = 0; k < (int)sc.size(); ++k) {
            if (!((changed[k >> 5] >> (k & 31)) & 1u)) continue;
            const int v = sc[k];
            std::memcpy(m->h_dom.data() + m->off[v], newDom + ld[k], (size_t)m->nw[v] * sizeof(uint32_t));
            mark_var(m, v, self, &q);
        }
    }
    return CT_OK;
}

extern "C" int ct_model_get_domains(ct_model* m, uint32_t* words_host) {
    if (!m || !words_host) {
        ct_set_error("ct_model_get_domains: null argument");
        return CT_ERR_ARG;
    }
    std::memcpy(words_host, m->h_dom.data(), (size_t)m->DWg * sizeof(uint32_t));
    return CT_OK;
}

extern "C" int ct_model_set_domains(ct_model* m, const uint32_t* words_host) {
    if (!m || !words_host) {
        ct_set_error("ct_model_set_domains: null argument");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_model_set_domains: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    for (int q = 0; q < m->DWg; ++q) {
        if (words_host[q] & ~m->h_dom[q]) {
            ct_set_error("ct_model_set_domains: domains may only shrink");
            return CT_ERR_STATE;
        }
    }
    for (int v = 0; v < m->nvars; ++v) {
        bool diff = false;
        for (int q = 0; q < m->nw[v]; ++q) diff |= words_host[m->off[v] + q] != m->h_dom[(size_t)m->off[v] + q];
        if (!diff) continue;
        const int st = set_var(m, v, words_host + m->off[v]);
        if (st != CT_OK) return st;
    }
    return CT_OK;
}

extern "C" int ct_model_save(ct_model* m, int* level_out) {
    if (!m) {
        ct_set_error("ct_model_save: null handle");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_model_save: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    const int L = (int)m->levels.size();
    int st;
    for (ct_table* tab : m->tables) {
        int l = 0;
        if ((st = ct_save(tab, &l)) != CT_OK) return st;
    }
    ct_model::Level lev;
    lev.dom = m->h_dom;
    lev.dirty = m->dirty;
    m->levels.push_back(std::move(lev));
    if (level_out) *level_out = L;
    return CT_OK;
}

extern "C" int ct_model_restore(ct_model* m, int level) {
    if (!m) {
        ct_set_error("ct_model_restore: null handle");
        return CT_ERR_ARG;
    }
    if (level < 0 || level >= (int)m->levels.size()) {
        ct_set_error("ct_model_restore: level %d not in [0, %d)", level, (int)m->levels.size());
        return CT_ERR_LEVEL;
    }
    // One launch undoes the trails of every table that changed since the level.
    RestoreBatch B;
    B.n = 0;
    for (int t = 0; t < (int)m->tables.size(); ++t) {
        RestoreDesc d{};
        const int need = ct_table_restore_prepare(m->tables[t], level, &d);
        if (need < 0) return need;
        if (!need) continue;
        if (!m->batchReady) {
            // no device copies of the tables yet: restore through the table itself
            const int r = ct_table_restore_device(m->tables[t], d);
            if (r != CT_OK) return r;
            continue;
        }
        if (ct_table_version(m->tables[t]) != m->tabVersion[t]) {
            CT_CUDA(cudaMemcpyAsync(m->d_tabs + t, &ct_table_dev(m->tables[t]), sizeof(TableDev),
                                    cudaMemcpyHostToDevice, m->stream));
            m->tabVersion[t] = ct_table_version(m->tables[t]);
        }
        d.table = t;
        B.d[B.n++] = d;
        if (B.n == kRestoreBatch) {
            CT_CUDA(launch_restore_batch(m->d_tabs, B, m->stream));
            B.n = 0;
        }
    }
    CT_CUDA(launch_restore_batch(m->d_tabs, B, m->stream));
    // The host copy is authoritative; the device copy follows lazily.
    m->h_dom = m->levels[level].dom;
    m->domStale = true;
    m->dirty = m->levels[level].dirty;
    m->levels.resize(level);
    m->failed = false;
    return CT_OK;
}

namespace {

struct Dfs {
    ct_model* m;
    int64_t limit;
    bool countAll;
    bool usePolicy = true;
    ct_branch_hook hook = nullptr;
    void* ctx = nullptr;
    int64_t traceN = 0;
    ct_search_stats st{};
    int32_t* firstSol;
    bool haveFirst = false;
    bool stop = false;
    bool hitLimit = false;

    // Returns CT_OK or a negative error.
    int node(int depth) {
        if (limit > 0 && st.nodes >= limit) {
            stop = true;
            hitLimit = true;
            return CT_OK;
        }
        st.nodes += 1;
        if (depth > st.max_depth) st.max_depth = depth;
        const int r = ct_model_propagate(m);
        if (r < 0) return r;
        if (r == CT_INFEASIBLE) {
            st.fails += 1;
            return CT_OK;
        }
        // First-fail (smallest domain among unfixed variables, ties to the lowest
        // index) or the policy's best-scored unfixed variable.
        int x = -1;
        const int ps = ct_model_pick_var(m, usePolicy, &x);
        if (ps != CT_OK) return ps;
        if (x < 0) {
            st.solutions += 1;
            if (!haveFirst) {
                haveFirst = true;
                if (firstSol) {
                    for (int v = 0; v < m->nvars; ++v) {
                        int a = 0;
                        for (int q = 0; q < m->nw[v]; ++q) {
                            const uint32_t w = m->h_dom[(size_t)m->off[v] + q];
                            if (w) {
                                a = q * 32 + __builtin_ctz(w);
                                break;
                            }
                        }
                        firstSol[v] = m->lo[v] + a;
                    }
                }
            }
            if (!countAll) stop = true;
            return CT_OK;
        }
        if (m->trace && traceN < m->traceCap) m->trace[traceN] = x;
        ++traceN;
        if (hook) {
            const int hs = hook(ctx, m);
            if (hs != CT_OK) return hs;
        }
        // Value: the minimum of dom(x).
        const int nwx = m->nw[x];
        std::vector<uint32_t> cur(m->h_dom.begin() + m->off[x], m->h_dom.begin() + m->off[x] + nwx);
        int a = 0;
        for (int q = 0; q < nwx; ++q) {
            if (cur[q]) {
                a = q * 32 + __builtin_ctz(cur[q]);
                break;
            }
        }
        std::vector<uint32_t> left(nwx, 0u), right(cur);
        left[a >> 5] = 1u << (a & 31);
        right[a >> 5] &= ~(1u << (a & 31));
        for (int branch = 0; branch < 2; ++branch) {
            int L = 0;
            int rc = ct_model_save(m, &L);
            if (rc != CT_OK) return rc;
            rc = set_var(m, x, branch == 0 ? left.data() : right.data());
            if (rc == CT_OK) rc = node(depth + 1);
            const int rr = ct_model_restore(m, L);
            if (rc != CT_OK) return rc;
            if (rr != CT_OK) return rr;
            if (stop) return CT_OK;
        }
        return CT_OK;
    }
};

}  // namespace

int ct_model_dfs(ct_model* m, int64_t node_limit, bool countAll, bool usePolicy, ct_search_stats* out,
                 int32_t* first_solution, ct_branch_hook hook, void* ctx) {
    if (!m || !out) {
        ct_set_error("ct_search_dfs: null argument");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_search_dfs: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t p0 = m->propagations;
    Dfs d;
    d.m = m;
    d.limit = node_limit;
    d.countAll = countAll;
    d.usePolicy = usePolicy;
    d.hook = hook;
    d.ctx = ctx;
    d.firstSol = first_solution;
    int L0 = 0;
    int st = ct_model_save(m, &L0);
    if (st != CT_OK) return st;
    st = d.node(0);
    const int rr = ct_model_restore(m, L0);
    if (st != CT_OK) return st;
    if (rr != CT_OK) return rr;
    CT_CUDA(cudaStreamSynchronize(m->stream));
    d.st.complete = d.hitLimit ? 0 : 1;
    d.st.propagations = m->propagations - p0;
    d.st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = d.st;
    if (m->trace && m->traceCount && !hook) *m->traceCount = std::min(d.traceN, m->traceCap);
    return CT_OK;
}

extern "C" int ct_search_dfs(ct_model* m, int64_t node_limit, int count_all, ct_search_stats* out,
                             int32_t* first_solution) {
    return ct_model_dfs(m, node_limit, count_all != 0, true, out, first_solution, nullptr, nullptr);
}

extern "C" int ct_model_features(ct_model* m, float* features_host) {
    if (!m || !features_host) {
        ct_set_error("ct_model_features: null argument");
        return CT_ERR_ARG;
    }
    if (m->failed) {
        ct_set_error("ct_model_features: the model failed; restore a level first");
        return CT_ERR_STATE;
    }
    int st = ensure_features(m);
    if (st == CT_OK) st = sync_dom(m);
    if (st == CT_OK) st = ct_feat_compute(m->fview, m->d_tabs, m->d_dom, nullptr, m->stream);
    if (st != CT_OK) return st;
    CT_CUDA(cudaMemcpyAsync(features_host, m->fview->feat, (size_t)m->nvars * kNF * sizeof(float),
                            cudaMemcpyDeviceToHost, m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    return CT_OK;
}

extern "C" int ct_model_get_stats(ct_model* m, ct_model_stats* out) {
    if (!m || !out) {
        ct_set_error("ct_model_get_stats: null argument");
        return CT_ERR_ARG;
    }
    *out = m->stats;
    if (m->batchReady && m->md.phaseNs) {
        uint64_t ns[kModelPhases];
        CT_CUDA(cudaMemcpyAsync(ns, m->md.phaseNs, sizeof(ns), cudaMemcpyDeviceToHost, m->stream));
        CT_CUDA(cudaStreamSynchronize(m->stream));
        for (int p = 0; p < kModelPhases; ++p) out->phase_seconds[p] = 1e-9 * (double)ns[p];
    }
    return CT_OK;
}

extern "C" int ct_model_reset_stats(ct_model* m) {
    if (!m) {
        ct_set_error("ct_model_reset_stats: null handle");
        return CT_ERR_ARG;
    }
    m->stats = ct_model_stats{};
    if (m->batchReady && m->md.phaseNs)
        CT_CUDA(cudaMemsetAsync(m->md.phaseNs, 0, kModelPhases * sizeof(uint64_t), m->stream));
    return CT_OK;
}

extern "C" int ct_model_set_policy(ct_model* m, ct_mlp* policy) {
    if (!m) {
        ct_set_error("ct_model_set_policy: null handle");
        return CT_ERR_ARG;
    }
    m->policy = policy;
    return CT_OK;
}

extern "C" int ct_model_set_trace(ct_model* m, int32_t* decisions_host, int64_t capacity, int64_t* count_host) {
    if (!m || capacity < 0) {
        ct_set_error("ct_model_set_trace: bad argument");
        return CT_ERR_ARG;
    }
    m->trace = decisions_host;
    m->traceCap = decisions_host ? capacity : 0;
    m->traceCount = count_host;
    return CT_OK;
}

extern "C" int ct_model_destroy(ct_model* m) {
    if (!m) return CT_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    ct_batch_free(m->bsearch);  // the clones share the tables' supports: freed first
    if (m->fview) {
        ct_feat_view_free(m->fview);
        delete m->fview;
    }
    for (ct_table* t : m->tables) ct_destroy(t);
    for (int32_t* p : m->d_tabOff) cudaFree(p);
    if (m->d_dom && !m->domInBlk) cudaFree(m->d_dom);
    if (m->h_stage) cudaFreeHost(m->h_stage);
    for (void* p : m->allocs) cudaFree(p);
    if (m->h_blk) cudaFreeHost(m->h_blk);
    if (m->h_mstatus) cudaFreeHost(m->h_mstatus);
    if (m->ownStream && m->stream) cudaStreamDestroy(m->stream);
    cudaGetLastError();
    delete m;
    return CT_OK;
}
