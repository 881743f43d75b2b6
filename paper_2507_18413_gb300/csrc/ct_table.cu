// ct_table.cu -- host side of one table constraint: construction of the
// device layout (Sec. 3 constructor, Sec. 4 device copies), propagation calls,
// backtrack levels and inspection.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "ct_table.cuh"

using namespace ctk;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void ct_set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int ct_cuda_fail(cudaError_t e, const char* what) {
    ct_set_error("%s: %s", what, cudaGetErrorString(e));
    return CT_ERR_CUDA;
}

extern "C" const char* ct_last_error(void) { return g_err.c_str(); }

extern "C" const char* ct_status_string(int s) {
    switch (s) {
        case CT_OK: return "CT_OK";
        case CT_INFEASIBLE: return "CT_INFEASIBLE";
        case CT_ERR_ARG: return "CT_ERR_ARG";
        case CT_ERR_OOM: return "CT_ERR_OOM";
        case CT_ERR_CUDA: return "CT_ERR_CUDA";
        case CT_ERR_STATE: return "CT_ERR_STATE";
        case CT_ERR_TIMEOUT: return "CT_ERR_TIMEOUT";
        case CT_ERR_LEVEL: return "CT_ERR_LEVEL";
        default: return "CT_UNKNOWN";
    }
}

extern "C" int ct_version(void) { return 10000; }

extern "C" int ct_read_ceiling(const void* dev_buf, int64_t bytes, void* cuda_stream, float* ms_out) {
    if (!dev_buf || bytes <= 0 || (bytes & 15) || (reinterpret_cast<uintptr_t>(dev_buf) & 15)) {
        ct_set_error("ct_read_ceiling: a 16-byte aligned buffer and a positive multiple of 16 bytes");
        return CT_ERR_ARG;
    }
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    if (ms_out) {
        e = cudaEventCreate(&ev[0]);
        if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    }
    if (e == cudaSuccess) e = ctk::launch_read_ceiling(static_cast<const uint4*>(dev_buf), (size_t)(bytes / 16), s);
    if (ms_out && e == cudaSuccess) {
        e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, ev[0], ev[1]);
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) {
        ct_set_error("ct_read_ceiling: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    return CT_OK;
}


namespace {

// ---------------------------------------------------------------------------
// device buffers of tables: every buffer a table owns (ct_create's buffers,
// the trail and the level stack) is allocated and freed here, with the test
// hooks ct_debug_*: guard regions around each buffer, a countdown that makes
// one allocation fail, and the bytes held, counted by the allocator itself
// ---------------------------------------------------------------------------
constexpr size_t kGuardBytes = 256;       // before and after a guarded buffer (keeps its 256-byte alignment)
constexpr unsigned char kGuardFill = 0xA5;
struct DevBuf {
    size_t bytes;
    bool guarded;
};
std::mutex g_bufMu;
std::unordered_map<void*, DevBuf> g_bufs;  // buffer as the table sees it -> size
int64_t g_bufBytes = 0;
bool g_guardNew = false;                   // ct_debug_guard_buffers
long long g_failAfter = -1;                // ct_debug_fail_alloc: allocations left before one fails

cudaError_t table_malloc(void** p, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_bufMu);
    *p = nullptr;
    if (g_failAfter >= 0) {
        if (g_failAfter == 0) {
            g_failAfter = -1;
            return cudaErrorMemoryAllocation;
        }
        --g_failAfter;
    }
    const bool guarded = g_guardNew;
    char* base = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&base), bytes + (guarded ? 2 * kGuardBytes : 0));
    if (e != cudaSuccess) return e;
    if (guarded) {
        e = cudaMemset(base, kGuardFill, kGuardBytes);
        if (e == cudaSuccess) e = cudaMemset(base + kGuardBytes + bytes, kGuardFill, kGuardBytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the guards are set before any use
        if (e != cudaSuccess) {
            cudaFree(base);
            return e;
        }
    }
    void* user = base + (guarded ? kGuardBytes : 0);
    g_bufs[user] = DevBuf{bytes, guarded};
    g_bufBytes += (int64_t)bytes;
    *p = user;
    return cudaSuccess;
}

void table_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_bufMu);
    const auto it = g_bufs.find(p);
    if (it == g_bufs.end()) {
        cudaFree(p);
        return;
    }
    g_bufBytes -= (int64_t)it->second.bytes;
    cudaFree(static_cast<char*>(p) - (it->second.guarded ? kGuardBytes : 0));
    g_bufs.erase(it);
}

template <typename T>
int dalloc(ct_table* ct, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    const cudaError_t e = table_malloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    ct->allocs.push_back(q);
    ct->deviceBytes += (int64_t)bytes;
    *p = static_cast<T*>(q);
    return CT_OK;
}

template <typename T>
int upload(ct_table* ct, T* dst, const std::vector<T>& src) {
    if (src.empty()) return CT_OK;
    CT_CUDA(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, ct->stream));
    return CT_OK;
}

int sync(ct_table* ct) {
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    return CT_OK;
}

// Grow the trail so that `need` entries fit.
// The event ring of ct_options.profile (created once, on first use).
int create_events(ct_table* ct) {
    ct->ev.assign(2 * ct_table::kEvRing, nullptr);
    for (auto& e : ct->ev) CT_CUDA(cudaEventCreate(&e));
    return CT_OK;
}

int ensure_trail(ct_table* ct, int64_t need) {
    if (need <= ct->trailCap) return CT_OK;
    if (need > 0x7fffffffLL) {
        ct_set_error("trail would exceed 2^31 entries");
        return CT_ERR_OOM;
    }
    int64_t cap = std::max<int64_t>(need, 2LL * ct->trailCap);
    if (cap > 0x7fffffffLL) cap = 0x7fffffffLL;
    int2* nk = nullptr;
    uint4* no = nullptr;
    cudaError_t e = table_malloc(reinterpret_cast<void**>(&nk), (size_t)cap * sizeof(int2));
    if (e == cudaSuccess) e = table_malloc(reinterpret_cast<void**>(&no), (size_t)cap * sizeof(uint4));
    if (e != cudaSuccess) {
        cudaGetLastError();
        table_free(nk);
        ct_set_error("trail growth to %lld entries: %s", (long long)cap, cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    if (ct->trailTop > 0) {
        CT_CUDA(cudaMemcpyAsync(nk, ct->dev.trailKey, (size_t)ct->trailTop * sizeof(int2), cudaMemcpyDeviceToDevice,
                                ct->stream));
        CT_CUDA(cudaMemcpyAsync(no, ct->dev.trailOld, (size_t)ct->trailTop * sizeof(uint4),
                                cudaMemcpyDeviceToDevice, ct->stream));
    }
    int32_t capi = (int32_t)cap;
    CT_CUDA(cudaMemcpyAsync(&ct->dev.ctrl->trail_cap, &capi, sizeof(int32_t), cudaMemcpyHostToDevice, ct->stream));
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    if (!ct->trailInArena) {
        table_free(ct->dev.trailKey);
        table_free(ct->dev.trailOld);
    }
    ct->trailInArena = false;
    ct->deviceBytes += (cap - ct->trailCap) * (int64_t)(sizeof(int2) + sizeof(uint4));
    ct->dev.trailKey = nk;
    ct->dev.trailOld = no;
    ct->trailCap = (int)cap;
    ct->version++;
    return CT_OK;
}

int ensure_levels(ct_table* ct, int need) {
    if (need <= ct->levelCap) return CT_OK;
    const int cap = std::max(need, 2 * ct->levelCap);
    uint32_t* ns = nullptr;
    uint32_t* nd = nullptr;
    cudaError_t e = table_malloc(reinterpret_cast<void**>(&ns), (size_t)cap * std::max(ct->nseg, 1) * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = table_malloc(reinterpret_cast<void**>(&nd), (size_t)cap * std::max(ct->DW, 1) * sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        table_free(ns);
        ct_set_error("level stack growth: %s", cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    const int used = (int)ct->levels.size();
    if (used > 0) {
        CT_CUDA(cudaMemcpyAsync(ns, ct->dev.levelSeg, (size_t)used * ct->nseg * sizeof(uint32_t),
                                cudaMemcpyDeviceToDevice, ct->stream));
        CT_CUDA(cudaMemcpyAsync(nd, ct->dev.levelDom, (size_t)used * ct->DW * sizeof(uint32_t),
                                cudaMemcpyDeviceToDevice, ct->stream));
    }
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    if (!ct->levelsInArena) {
        table_free(ct->dev.levelSeg);
        table_free(ct->dev.levelDom);
    }
    ct->levelsInArena = false;
    ct->deviceBytes += (int64_t)(cap - ct->levelCap) * (ct->nseg * 4 + ct->DW * 4);
    ct->dev.levelSeg = ns;
    ct->dev.levelDom = nd;
    ct->levelCap = cap;
    ct->version++;
    return CT_OK;
}

void free_table(ct_table* ct) {
    if (!ct) return;
    if (ct->stream) cudaStreamSynchronize(ct->stream);
    for (void* p : ct->allocs) table_free(p);
    if (!ct->trailInArena) {
        table_free(ct->dev.trailKey);
        table_free(ct->dev.trailOld);
    }
    if (!ct->levelsInArena) {
        table_free(ct->dev.levelSeg);
        table_free(ct->dev.levelDom);
    }
    if (ct->h_status) cudaFreeHost(ct->h_status);
    if (ct->h_curr) cudaFreeHost(ct->h_curr);
    for (auto& e : ct->ev)
        if (e) cudaEventDestroy(e);
    if (ct->ownStream && ct->stream) cudaStreamDestroy(ct->stream);
    cudaGetLastError();
    delete ct;
}

int build(ct_table* ct, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples, int64_t t,
          const ct_options* opt, bool negative) {
    const int n = ct->arity;
    ct->lo.assign(dom_lo, dom_lo + n);
    ct->size.assign(dom_size, dom_size + n);
    ct->nw.resize(n);
    ct->ld.resize(n);
    ct->row0.resize(n + 1);
    int DW = 0, R = 0;
    for (int i = 0; i < n; ++i) {
        ct->nw[i] = (ct->size[i] + 31) / 32;
        ct->ld[i] = DW;
        DW += ct->nw[i];
        ct->row0[i] = R;
        R += ct->size[i];
    }
    ct->row0[n] = R;
    ct->DW = DW;
    ct->R = R;
    ct->nChW = (n + 31) / 32;
    ct->rowVar.resize(R);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < ct->size[i]; ++a) ct->rowVar[ct->row0[i] + a] = i;

    // Retained tuples: every value inside its initial domain or a wildcard
    // (input order kept).
    std::vector<int64_t> keep;
    keep.reserve((size_t)t);
    int64_t nShort = 0;
    for (int64_t j = 0; j < t; ++j) {
        const int32_t* tu = tuples + j * n;
        bool ok = true, star = false;
        for (int i = 0; i < n && ok; ++i) {
            if (tu[i] == CT_STAR) {
                star = true;
                continue;
            }
            const int64_t off = (int64_t)tu[i] - ct->lo[i];
            ok = off >= 0 && off < ct->size[i];
        }
        if (ok) {
            keep.push_back(j);
            nShort += star;
        }
    }
    ct->shortTuples = nShort;
    if (negative) {
        // forbidden tuples: no wildcard, each counted once (the filter compares counts)
        if (nShort > 0) {
            ct_set_error("ct_create_negative: wildcards are not allowed in a negative table");
            return CT_ERR_ARG;
        }
        std::vector<std::pair<std::vector<int32_t>, int64_t>> keyed;
        keyed.reserve(keep.size());
        for (int64_t j : keep) keyed.push_back({std::vector<int32_t>(tuples + j * n, tuples + j * n + n), j});
        std::stable_sort(keyed.begin(), keyed.end(),
                         [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t q = 1; q < keyed.size(); ++q)
            if (keyed[q].first == keyed[q - 1].first) keyed[q].second = -1 - keyed[q].second;
        std::vector<int64_t> drop;
        for (const auto& kv : keyed)
            if (kv.second < 0) drop.push_back(-1 - kv.second);
        std::sort(drop.begin(), drop.end());
        std::vector<int64_t> kept2;
        kept2.reserve(keep.size());
        for (int64_t j : keep)
            if (!std::binary_search(drop.begin(), drop.end(), j)) kept2.push_back(j);
        keep.swap(kept2);
        if (keep.empty()) {
            ct_set_error("ct_create_negative: a negative table needs at least one tuple inside the domains");
            return CT_ERR_ARG;
        }
        if (!(n <= kLocalMaxArity && ct->DW <= kLocalMaxDW && ct->R <= kCodeCap)) {
            ct_set_error("ct_create_negative: arity <= %d, <= %d domain words and <= %d values", kLocalMaxArity,
                         kLocalMaxDW, kCodeCap);
            return CT_ERR_ARG;
        }
        ct->negative = true;
    }
    ct->t = (int64_t)keep.size();
    ct->W = (ct->t + 31) / 32;
    ct->W4 = (ct->W + 3) / 4;
    ct->profile = opt && opt->profile;
    ct->copyState = opt && opt->copy_state;
    if (ct->t == 0) {
        ct->empty = true;
        return CT_INFEASIBLE;
    }
    if (ct->W4 > 0x3fffffffLL) {
        ct_set_error("too many tuples");
        return CT_ERR_ARG;
    }
    const int64_t W4 = ct->W4;
    ct->S = 32;
    ct->nseg = (int)((W4 + 31) / 32);
    ct->localPlan = n <= kLocalMaxArity && DW <= kLocalMaxDW && R <= kCodeCap;

    // supports rows (Sec. 2), value-major, 16-byte aligned rows of W4 chunks
    // (a short tuple is in every row of its wildcard positions; the delta rows
    // hold only the tuples whose component equals the row's value)
    const size_t rowWords = (size_t)W4 * 4;
    std::vector<uint32_t> hsup((size_t)R * rowWords, 0u);
    std::vector<uint32_t> hdel;
    if (nShort > 0) hdel.assign((size_t)R * rowWords, 0u);
    for (int64_t jj = 0; jj < ct->t; ++jj) {
        const int32_t* tu = tuples + keep[(size_t)jj] * n;
        const uint32_t bit = 1u << (jj & 31);
        const size_t word = (size_t)(jj >> 5);
        for (int i = 0; i < n; ++i) {
            if (tu[i] == CT_STAR) {
                for (int a = 0; a < ct->size[i]; ++a) hsup[(size_t)(ct->row0[i] + a) * rowWords + word] |= bit;
                continue;
            }
            const int row = ct->row0[i] + (tu[i] - ct->lo[i]);
            hsup[(size_t)row * rowWords + word] |= bit;
            if (nShort > 0) hdel[(size_t)row * rowWords + word] |= bit;
        }
    }
    std::vector<int32_t> hres(R, 0);
    for (int r = 0; r < R; ++r) {
        const uint32_t* row = hsup.data() + (size_t)r * rowWords;
        for (int64_t c = 0; c < W4; ++c) {
            if (row[c * 4] | row[c * 4 + 1] | row[c * 4 + 2] | row[c * 4 + 3]) {
                hres[r] = (int32_t)c;
                break;
            }
        }
    }
    // currTable: every retained tuple is valid under the initial domains.
    std::vector<uint32_t> hcurr(rowWords, 0u);
    for (int64_t w = 0; w < ct->W; ++w) {
        const int64_t rem = ct->t - w * 32;
        hcurr[(size_t)w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    // Non-zero index: every chunk below W4 holds a retained tuple at creation.
    std::vector<uint32_t> hmask(ct->nseg, 0u);
    for (int s = 0; s < ct->nseg; ++s) {
        const int64_t left = W4 - (int64_t)s * 32;
        hmask[s] = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
    }
    std::vector<uint32_t> hdom(DW, 0u);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < ct->size[i]; ++a) hdom[ct->ld[i] + a / 32] |= 1u << (a % 32);

    TableDev& d = ct->dev;
    int st;
    uint4* sup = nullptr;
    int32_t *rowVar = nullptr, *varRow0 = nullptr, *varNW = nullptr, *varLD = nullptr;
    if ((st = dalloc(ct, &sup, (size_t)R * W4)) != CT_OK) return st;
    uint4* supDel = sup;
    if (nShort > 0 && (st = dalloc(ct, &supDel, (size_t)R * W4)) != CT_OK) return st;
    // currTable and lastpos are padded to whole 32-chunk segments.
    const size_t padChunks = (size_t)ct->nseg * 32;
    if ((st = dalloc(ct, &d.curr, padChunks)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.segMask, (size_t)ct->nseg)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.lastpos, padChunks)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.residue, (size_t)R)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.lastDom, (size_t)DW)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.ctrl, 1)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.codes, (size_t)R)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.planK, (size_t)n)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.planRowOff, (size_t)n)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.varSup, (size_t)n)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.other, (size_t)n)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.hardRow, (size_t)R)) != CT_OK) return st;
    if ((st = dalloc(ct, &d.foundChunk, (size_t)R)) != CT_OK) return st;
    if ((st = dalloc(ct, &rowVar, (size_t)R)) != CT_OK) return st;
    if ((st = dalloc(ct, &varRow0, (size_t)n + 1)) != CT_OK) return st;
    if ((st = dalloc(ct, &varNW, (size_t)n)) != CT_OK) return st;
    if ((st = dalloc(ct, &varLD, (size_t)n)) != CT_OK) return st;
    ct->statusInts = (size_t)kStatusHdr + ct->nChW + DW;
    if ((st = dalloc(ct, &ct->d_domScratch, (size_t)DW)) != CT_OK) return st;
    d.sup = sup;
    d.supDelta = supDel;
    d.negative = ct->negative ? 1 : 0;
    d.shard = (opt && opt->shard) ? 1 : 0;
    d.rowVar = rowVar;
    d.varRow0 = varRow0;
    d.varNW = varNW;
    d.varLD = varLD;
    d.arity = n;
    d.R = R;
    d.W4 = (int32_t)W4;
    d.nseg = ct->nseg;
    d.S = ct->S;
    d.DW = DW;
    d.nChangedWords = ct->nChW;
    d.useResidues = (opt && opt->no_residues) ? 0 : 1;
    d.warpPlan = (!ct->negative && n <= 32) ? 1 : 0;
    for (int i = 0; i < n; ++i)
        if (ct->nw[i] > kWarpPlanWords) d.warpPlan = 0;
    for (int i = 0; i < n && i < kParamArity; ++i) {
        d.pNW[i] = ct->nw[i];
        d.pLD[i] = ct->ld[i];
        d.pRow0[i] = ct->row0[i];
    }
    ct->live = (int)W4;

    // The status block lives in mapped host memory: the kernel's last CTA writes
    // it directly and the host reads it after the stream synchronises.
    if (cudaHostAlloc((void**)&ct->h_status, ct->statusInts * sizeof(int32_t), cudaHostAllocMapped) !=
        cudaSuccess) {
        cudaGetLastError();
        ct->h_status = nullptr;
        ct_set_error("cudaHostAlloc of the status block failed");
        return CT_ERR_OOM;
    }
    std::memset(ct->h_status, 0, ct->statusInts * sizeof(int32_t));
    CT_CUDA(cudaHostGetDevicePointer((void**)&d.statusBlk, ct->h_status, 0));
    {
        // 16 loads in flight per lane at 2 CTAs per SM. With the row list of a
        // segment cut over up to kMaxSplit warps of a CTA, every segment can
        // keep a whole CTA busy: one CTA per segment (a long row list then
        // spreads over the whole grid), capped at residency, and at least one
        // warp per two values for the probes.
        ct->maxSplit = (opt && opt->no_split) ? 1 : kMaxSplit;
        ct->early = !(opt && opt->no_early_filter);
        const int narrow = (ct->localPlan ? 1 : 0);
        // more segments than one wave of warps at 2 CTAs per SM: 8 loads at 3 CTAs per SM
        const int maxNarrow = max_coresident_blocks(narrow);
        ct->variant = (ct->nseg > maxNarrow * kWarps) ? (narrow | 2) : narrow;
        const int maxCo = max_coresident_blocks(ct->variant);
        if (maxCo <= 0) {
            ct_set_error("ct_create: the propagation kernel cannot be made resident on this device");
            return CT_ERR_CUDA;
        }
        int want = (ct->nseg * ct->maxSplit + kWarps - 1) / kWarps;
        want = std::max(want, (R + 2 * kWarps - 1) / (2 * kWarps));
        if (opt && opt->grid_blocks > 0) want = opt->grid_blocks;
        ct->grid = std::max(1, std::min(want, maxCo));
    }

    CT_CUDA(cudaMemcpyAsync(sup, hsup.data(), hsup.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, ct->stream));
    if (nShort > 0)
        CT_CUDA(cudaMemcpyAsync(supDel, hdel.data(), hdel.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                ct->stream));
    CT_CUDA(cudaMemsetAsync(d.curr, 0, padChunks * sizeof(uint4), ct->stream));
    CT_CUDA(cudaMemcpyAsync(d.curr, hcurr.data(), hcurr.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            ct->stream));
    if ((st = upload(ct, d.segMask, hmask)) != CT_OK) return st;
    CT_CUDA(cudaMemsetAsync(d.lastpos, 0xff, padChunks * sizeof(int32_t), ct->stream));
    if ((st = upload(ct, d.residue, hres)) != CT_OK) return st;
    if ((st = upload(ct, d.lastDom, hdom)) != CT_OK) return st;
    if ((st = upload(ct, rowVar, ct->rowVar)) != CT_OK) return st;
    if ((st = upload(ct, varRow0, ct->row0)) != CT_OK) return st;
    if ((st = upload(ct, varNW, ct->nw)) != CT_OK) return st;
    if ((st = upload(ct, varLD, ct->ld)) != CT_OK) return st;
    CT_CUDA(cudaMemsetAsync(d.other, 0, (size_t)n * sizeof(unsigned long long), ct->stream));

    Ctrl c{};
    c.status = CT_OK;
    c.trail_top = 0;
    c.cur_mark = -1;
    c.trail_cap = 0;
    CT_CUDA(cudaMemcpyAsync(d.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, ct->stream));
    if ((st = sync(ct)) != CT_OK) return st;
    if ((st = ensure_levels(ct, 8)) != CT_OK) return st;
    if (ct->profile) {
        if ((st = create_events(ct)) != CT_OK) return st;
    }
    return sync(ct);
}

void fill_stats(ct_table* ct) {
    const int32_t* h = ct->h_status;
    ct_call_stats& s = ct->last;
    s.status = h[kSlotStatus];
    s.changed_vars = h[kSlotNval];
    s.delta_vars = h[kSlotNdelta];
    s.reset_vars = h[kSlotNreset];
    s.rows_ored = h[kSlotRowsOred];
    s.sup_vars = h[kSlotNsup];
    s.residue_hits = h[kSlotHits];
    s.local_found = h[kSlotLocal];
    s.hard = h[kSlotHard];
    s.windows = h[kSlotWindows];
    s.pruned = h[kSlotPruned];
    s.trail_added = h[kSlotTrailAdded];
    s.live_chunks_in = (uint32_t)h[kSlotLiveIn];
    s.live_chunks_out = (uint32_t)h[kSlotLiveOut];
    s.live_words_in = (uint32_t)h[kSlotWordsIn];
    // Algorithmic bytes (what CT itself must move, 4-byte words): updateTable
    // reads k rows and currTable and writes currTable over the N live words;
    // filterDomains reads one word per residue hit, the windows it probes and
    // the whole live table for every value scanned in full.
    s.update_bytes = s.rows_ored > 0 ? 4LL * s.live_words_in * (s.rows_ored + 2) : 0;
    s.filter_bytes = 4LL * s.residue_hits + 4LL * 128 * s.windows + 16LL * s.hard * s.live_chunks_out;
    s.phase_ns[0] = h[kSlotT1];
    s.phase_ns[1] = h[kSlotT2];
    s.phase_ns[2] = h[kSlotT3];
    s.phase_ns[3] = h[kSlotT4];
    s.early_filter = h[kSlotEarly];
}

}  // namespace

// ---------------------------------------------------------------------------
// internal entry points for the model
// ---------------------------------------------------------------------------
namespace {

// Read the oldest pending event pair into the profile (waits for it).
int drain_event(ct_table* ct) {
    if (ct->evPending == 0) return CT_OK;
    const int slot = (ct->evNext - ct->evPending + ct_table::kEvRing) % ct_table::kEvRing;
    float a = 0.f;
    CT_CUDA(cudaEventSynchronize(ct->ev[2 * slot + 1]));
    CT_CUDA(cudaEventElapsedTime(&a, ct->ev[2 * slot], ct->ev[2 * slot + 1]));
    ct->prof.kernel_ms += a;
    ct->evPending -= 1;
    return CT_OK;
}

// copy_state ablation: the host copy of currTable, (re)read from the device.
int fetch_host_curr(ct_table* ct) {
    const size_t bytes = (size_t)ct->W4 * sizeof(uint4);
    if (!ct->h_curr && cudaHostAlloc((void**)&ct->h_curr, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        ct->h_curr = nullptr;
        ct_set_error("copy_state: pinned host copy of currTable");
        return CT_ERR_OOM;
    }
    CT_CUDA(cudaMemcpyAsync(ct->h_curr, ct->dev.curr, bytes, cudaMemcpyDeviceToHost, ct->stream));
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    return CT_OK;
}

int drain_events(ct_table* ct) {
    int st = CT_OK;
    while (ct->evPending > 0 && (st = drain_event(ct)) == CT_OK) {
    }
    return st;
}

}  // namespace

// domHost (host memory, the table's packed layout; local-plan tables with at
// most kParamDomWords domain words): the domains travel in the kernel
// parameters instead of `dom`, which may then be null; the filtered domains
// are in the status block when the call returns.
int ct_table_propagate_on(ct_table* ct, uint32_t* dom, const int32_t* domOffDev, const int32_t* domOffHost,
                          uint32_t* changed, const uint32_t* domHost) {
    if (!ct || (!dom && !domHost)) {
        ct_set_error("ct_propagate: null argument");
        return CT_ERR_ARG;
    }
    if (ct->empty) {
        ct->last = ct_call_stats{};
        ct->last.status = CT_INFEASIBLE;
        ct->failed = true;
        return CT_INFEASIBLE;
    }
    if (ct->broken) {
        ct_set_error("ct_propagate: the table is unusable after a device-side timeout");
        return CT_ERR_TIMEOUT;
    }
    if (ct->failed) {
        ct_set_error("ct_propagate: the previous call failed; restore a level first");
        return CT_ERR_STATE;
    }
    int st;
    if (!ct->levels.empty() && (st = ensure_trail(ct, (int64_t)ct->trailTop + ct->W4)) != CT_OK) return st;
    cudaStream_t s = ct->stream;
    int32_t* h = ct->h_status;
    volatile int32_t* hv = h;
    const auto t0 = std::chrono::steady_clock::now();
    CallParams P{};
    P.mark = ct->levels.empty() ? -1 : ct->levels.back().mark;
    P.snapFrom = ct->pendingFrom;
    P.snapTo = (int)ct->levels.size();
    P.prevLive = ct->live;
    P.spinLimit = kBarrierSpinLimit;
    P.maxSplit = ct->maxSplit;
    P.early = ct->early ? 16 : 0;
    for (int i = 0; i < ct->arity && i < kParamArity; ++i) P.domOff[i] = domOffHost[i];
    if (domHost) {
        if (!ct->localPlan || ct->DW > kParamDomWords) {
            ct_set_error("ct_propagate: domains in parameters need a local plan and <= %d words", kParamDomWords);
            return CT_ERR_ARG;
        }
        P.domInParams = 1;
        std::memcpy(P.domWords, domHost, (size_t)ct->DW * sizeof(uint32_t));
    }
    hv[kSlotStatus] = kNoChunk;  // overwritten by the kernel's last CTA
    if (ct->armPolls) {
        // Test hook (ct_arm_wait_timeout): an arrival count 2^30 behind every
        // target of this call (base 0), so no barrier completes and every wait
        // runs out after armPolls polls.
        const uint32_t unreachable[2] = {0xC0000000u, 0u};  // bar_count, bar_base
        static_assert(offsetof(Ctrl, bar_base) == offsetof(Ctrl, bar_count) + sizeof(uint32_t), "adjacent words");
        CT_CUDA(cudaMemcpyAsync(&ct->dev.ctrl->bar_count, unreachable, sizeof(unreachable), cudaMemcpyHostToDevice, s));
        P.spinLimit = ct->armPolls;
        ct->armPolls = 0;
    }
    if (ct->copyState) {
        // the paper's propagators copy currTable to the device before each call
        if (!ct->h_curr && (st = fetch_host_curr(ct)) != CT_OK) return st;
        CT_CUDA(cudaMemcpyAsync(ct->dev.curr, ct->h_curr, (size_t)ct->W4 * sizeof(uint4), cudaMemcpyHostToDevice, s));
    }
    int evSlot = 0;
    if (ct->profile) {
        if (ct->evPending == ct_table::kEvRing && (st = drain_event(ct)) != CT_OK) return st;
        evSlot = ct->evNext;
        CT_CUDA(cudaEventRecord(ct->ev[2 * evSlot], s));
    }
    CT_CUDA(launch_propagate(ct->dev, ct->variant, ct->grid, dom, domOffDev, P, s));
    if (ct->profile) {
        CT_CUDA(cudaEventRecord(ct->ev[2 * evSlot + 1], s));
        ct->evNext = (ct->evNext + 1) % ct_table::kEvRing;
        ct->evPending += 1;
    }
    const auto t1 = std::chrono::steady_clock::now();
    ct->pendingFrom = (int)ct->levels.size();
    // Wait for the status word the kernel publishes last (bounded), then fall
    // back to a stream synchronisation to collect any CUDA error.
    // A kernel that returned without publishing (a barrier wait ran out) is
    // noticed when the stream has gone idle.
    bool seen = false;
    for (uint64_t it = 0;; ++it) {
        if (hv[kSlotStatus] != kNoChunk) {
            seen = true;
            break;
        }
        if ((it & 1023u) == 1023u) {
            if (cudaStreamQuery(s) == cudaSuccess) {
                seen = hv[kSlotStatus] != kNoChunk;
                break;
            }
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(kHostWaitMs)) break;
        }
    }
    if (!seen) CT_CUDA(cudaStreamSynchronize(s));
    if (ct->copyState) {
        // ... and back to the host after it
        CT_CUDA(cudaMemcpyAsync(ct->h_curr, ct->dev.curr, (size_t)ct->W4 * sizeof(uint4), cudaMemcpyDeviceToHost, s));
        CT_CUDA(cudaStreamSynchronize(s));
    }
    const auto t2 = std::chrono::steady_clock::now();
    int status = hv[kSlotStatus];
    if (status == kNoChunk) {
        // The kernel returned before publishing: a grid barrier timed out.
        Ctrl c{};
        CT_CUDA(cudaMemcpy(&c, ct->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
        status = c.status == CT_OK ? CT_ERR_TIMEOUT : c.status;
        c.bar_count = c.bar_base = 0;
        c.status = CT_OK;
        c.live = c.live_in = c.words_in = c.nhard = c.done = c.tuples = 0u;
        c.nscan = 0;
        c.upd_done = 0u;
        CT_CUDA(cudaMemcpy(ct->dev.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice));
        ct->failed = true;
        ct->broken = true;
        ct->last = ct_call_stats{};
        ct->last.status = status;
        ct_set_error("ct_propagate: a device-side wait ran out (status %d)", status);
        return status;
    }
    fill_stats(ct);
    ct->trailTop = h[kSlotTrailTop];
    if (status == CT_OK) ct->live = h[kSlotLiveOut];
    if (ct->profile) {
        ct->prof.host_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        ct->prof.launch_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
        ct->prof.wait_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
        ct->prof.calls += 1;
        ct->prof.update_bytes += ct->last.update_bytes;
        ct->prof.filter_bytes += ct->last.filter_bytes;
        ct->prof.device_ms += ct->last.phase_ns[3] * 1e-6;
    }
    if (status == CT_INFEASIBLE) {
        ct->failed = true;
    } else if (status == CT_ERR_STATE) {
        ct_set_error("ct_propagate: a domain grew since the last call without a restore");
    } else if (status == CT_ERR_OOM) {
        ct->failed = true;
        ct_set_error("ct_propagate: trail overflow");
    } else if (status != CT_OK) {
        ct->failed = true;
        ct_set_error("ct_propagate: device status %d", status);
    }
    if (changed) {
        // The changed mask is only written when a value was pruned.
        if (status == CT_OK && h[kSlotPruned] > 0)
            std::memcpy(changed, h + kStatusHdr, (size_t)ct->nChW * sizeof(uint32_t));
        else
            std::memset(changed, 0, (size_t)ct->nChW * sizeof(uint32_t));
    }
    return status;
}

const int32_t* ct_table_status_host(const ct_table* ct) { return ct->h_status; }

// --- the batched network path (ct_model.cu) ---
int ct_table_is_empty(const ct_table* ct) { return ct->empty ? 1 : 0; }

int ct_table_grow_trail(ct_table* ct, int64_t need) { return ensure_trail(ct, need); }


namespace {

constexpr int kCloneLevels = 8;

int64_t clone_trail_entries(const ct_table* src) { return 2 * src->W4 + 64; }

size_t rnd256(size_t b) { return (std::max<size_t>(b, 1) + 255) & ~size_t(255); }

// Bytes of every dynamic buffer of a clone, in allocation order.
std::vector<size_t> clone_pieces(const ct_table* src) {
    const size_t padChunks = (size_t)src->nseg * 32;
    const size_t R = (size_t)src->R, n = (size_t)src->arity;
    const size_t tr = (size_t)clone_trail_entries(src);
    return {padChunks * sizeof(uint4), (size_t)src->nseg * 4, padChunks * 4, R * 4, (size_t)src->DW * 4, R * 4,
            n * 4, n * 4, n * 4, n * 8, R * 4, R * 4,
            (size_t)kCloneLevels * std::max(src->nseg, 1) * 4, (size_t)kCloneLevels * std::max(src->DW, 1) * 4,
            tr * sizeof(int2), tr * sizeof(uint4)};
}

}  // namespace

size_t ct_table_clone_bytes(const ct_table* src) {
    size_t b = 0;
    for (size_t p : clone_pieces(src)) b += rnd256(p);
    return b + 256;
}

// A table that shares `src`'s static buffers (supports rows and the layout
// tables, which stay owned by src) with dynamic buffers of its own (currTable,
// index, lastDom, residues, trail, levels), filled by launch_clone_state. Used
// for the independent search nodes of a batched search. With an arena the
// dynamic buffers, 8 levels and a first trail come out of it in one piece;
// a trail or level stack that outgrows them moves to its own allocation.
ct_table* ct_table_clone(const ct_table* src, cudaStream_t stream, DeviceArena* arena, Ctrl* ctrl, int* status) {
    *status = CT_ERR_ARG;
    if (!src || src->empty) return nullptr;
    ct_table* ct = new (std::nothrow) ct_table();
    if (!ct) {
        *status = CT_ERR_OOM;
        return nullptr;
    }
    ct->arity = src->arity;
    ct->lo = src->lo;
    ct->size = src->size;
    ct->nw = src->nw;
    ct->ld = src->ld;
    ct->row0 = src->row0;
    ct->rowVar = src->rowVar;
    ct->R = src->R;
    ct->t = src->t;
    ct->W = src->W;
    ct->W4 = src->W4;
    ct->nseg = src->nseg;
    ct->S = src->S;
    ct->grid = src->grid;
    ct->DW = src->DW;
    ct->nChW = src->nChW;
    ct->localPlan = src->localPlan;
    ct->variant = src->variant;
    ct->maxSplit = src->maxSplit;
    ct->early = src->early;
    ct->live = src->live;
    ct->stream = stream;
    ct->dev = src->dev;  // static pointers shared; dynamic ones replaced below
    TableDev& d = ct->dev;
    d.trailKey = nullptr;
    d.trailOld = nullptr;
    d.levelSeg = nullptr;
    d.levelDom = nullptr;
    d.statusBlk = src->dev.statusBlk;  // never written by the batched path; kept valid
    if (arena) {
        const std::vector<size_t> pc = clone_pieces(src);
        void* p[16];
        for (int i = 0; i < 16; ++i) {
            p[i] = arena->take(pc[i]);
            if (!p[i]) {
                free_table(ct);
                ct_set_error("clone arena exhausted");
                *status = CT_ERR_OOM;
                return nullptr;
            }
        }
        d.curr = static_cast<uint4*>(p[0]);
        d.segMask = static_cast<uint32_t*>(p[1]);
        d.lastpos = static_cast<int32_t*>(p[2]);
        d.residue = static_cast<int32_t*>(p[3]);
        d.lastDom = static_cast<uint32_t*>(p[4]);
        d.codes = static_cast<int32_t*>(p[5]);
        d.planK = static_cast<int32_t*>(p[6]);
        d.planRowOff = static_cast<int32_t*>(p[7]);
        d.varSup = static_cast<int32_t*>(p[8]);
        d.other = static_cast<unsigned long long*>(p[9]);
        d.hardRow = static_cast<int32_t*>(p[10]);
        d.foundChunk = static_cast<int32_t*>(p[11]);
        d.levelSeg = static_cast<uint32_t*>(p[12]);
        d.levelDom = static_cast<uint32_t*>(p[13]);
        d.trailKey = static_cast<int2*>(p[14]);
        d.trailOld = static_cast<uint4*>(p[15]);
        ct->levelCap = kCloneLevels;
        ct->levelsInArena = true;
        ct->trailCap = (int)clone_trail_entries(src);
        ct->trailInArena = true;
        int st = CT_OK;
        if (ctrl) d.ctrl = ctrl;
        else if ((st = dalloc(ct, &d.ctrl, 1)) != CT_OK) {
            free_table(ct);
            *status = st;
            return nullptr;
        }
        *status = CT_OK;
        return ct;
    }
    const size_t padChunks = (size_t)ct->nseg * 32;
    int st = CT_OK;
    if ((st = dalloc(ct, &d.curr, padChunks)) != CT_OK || (st = dalloc(ct, &d.segMask, (size_t)ct->nseg)) != CT_OK ||
        (st = dalloc(ct, &d.lastpos, padChunks)) != CT_OK || (st = dalloc(ct, &d.residue, (size_t)ct->R)) != CT_OK ||
        (st = dalloc(ct, &d.lastDom, (size_t)ct->DW)) != CT_OK || (st = dalloc(ct, &d.codes, (size_t)ct->R)) != CT_OK ||
        (st = dalloc(ct, &d.planK, (size_t)ct->arity)) != CT_OK ||
        (st = dalloc(ct, &d.planRowOff, (size_t)ct->arity)) != CT_OK ||
        (st = dalloc(ct, &d.varSup, (size_t)ct->arity)) != CT_OK ||
        (st = dalloc(ct, &d.other, (size_t)ct->arity)) != CT_OK ||
        (st = dalloc(ct, &d.hardRow, (size_t)ct->R)) != CT_OK || (st = dalloc(ct, &d.foundChunk, (size_t)ct->R)) != CT_OK) {
        free_table(ct);
        *status = st;
        return nullptr;
    }
    if (ctrl) d.ctrl = ctrl;
    else if ((st = dalloc(ct, &d.ctrl, 1)) != CT_OK) {
        free_table(ct);
        *status = st;
        return nullptr;
    }
    if ((st = ensure_levels(ct, kCloneLevels)) != CT_OK) {
        free_table(ct);
        *status = st;
        return nullptr;
    }
    *status = CT_OK;
    return ct;
}

int ct_table_trail_cap(const ct_table* ct) { return ct->trailCap; }

// Host side of a clone taking its source's state (the device side is
// launch_clone_state): empty trail, no levels, the source's live count.
void ct_table_adopt_state(ct_table* dst, const ct_table* src) {
    dst->live = src->live;
    dst->trailTop = 0;
    dst->levels.clear();
    dst->pendingFrom = 0;
    dst->failed = false;
}

int ct_table_live(const ct_table* ct) { return ct->live; }

void ct_table_free(ct_table* ct) { free_table(ct); }


int ct_table_depth(const ct_table* ct) { return (int)ct->levels.size(); }

int ct_table_restore_device(ct_table* ct, const RestoreDesc& d) {
    CT_CUDA(launch_restore(ct->dev, d.level, d.mark, d.top, -1, ct->stream));
    return CT_OK;
}

int ct_table_dom_words(const ct_table* ct) { return ct->DW; }
const int32_t* ct_table_var_ld(const ct_table* ct) { return ct->ld.data(); }
int ct_table_changed_words(const ct_table* ct) { return ct->nChW; }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

// Launch-shape autotuner: time trial propagations of every candidate shape
// (row loads in flight x CTA count) between a save and a restore, keep the
// fastest. Trials: a delta call (one value of the largest domain removed) and
// a reset call (every domain cut to a quarter); the score is the sum of their
// best-of-3 host-observed latencies (launch to published result).
int autotune(ct_table* ct) {
    if (ct->empty || ct->R < 1) return CT_OK;
    const int narrow = ct->localPlan ? 1 : 0;
    const int base = std::max((ct->nseg * ct->maxSplit + kWarps - 1) / kWarps, (ct->R + 2 * kWarps - 1) / (2 * kWarps));
    std::vector<std::pair<int, int>> cands;
    for (int wide = 0; wide < 2; ++wide) {
        const int var = narrow | (wide ? 2 : 0);
        const int maxCo = max_coresident_blocks(var);
        if (maxCo <= 0) continue;
        for (int g : {base / 4, base / 2, base, 2 * base, maxCo / 2, maxCo}) {
            g = std::max(1, std::min(g, maxCo));
            if (std::find(cands.begin(), cands.end(), std::make_pair(var, g)) == cands.end()) cands.push_back({var, g});
        }
    }
    if (cands.empty()) return CT_OK;
    // trial domains in the table's packed layout
    std::vector<uint32_t> full((size_t)ct->DW, 0u), delta, reset;
    int big = 0;
    for (int i = 0; i < ct->arity; ++i) {
        for (int a = 0; a < ct->size[i]; ++a) full[(size_t)ct->ld[i] + a / 32] |= 1u << (a % 32);
        if (ct->size[i] > ct->size[big]) big = i;
    }
    delta = full;
    reset = full;
    if (ct->size[big] > 1) delta[(size_t)ct->ld[big]] &= ~1u;
    for (int i = 0; i < ct->arity; ++i) {
        const int keep = std::max(1, ct->size[i] / 4);
        for (int a = keep; a < ct->size[i]; ++a) reset[(size_t)ct->ld[i] + a / 32] &= ~(1u << (a % 32));
    }
    const int saveVar = ct->variant, saveGrid = ct->grid;
    const bool saveProfile = ct->profile;
    ct->profile = false;
    int L = 0;
    int st = ct_save(ct, &L);
    if (st != CT_OK) return st;
    double best = 1e30;
    int bestVar = saveVar, bestGrid = saveGrid;
    for (const auto& c : cands) {
        ct->variant = c.first;
        ct->grid = c.second;
        double score = 0.0;
        for (const std::vector<uint32_t>* trial : {&delta, &reset}) {
            double tmin = 1e30;
            for (int rep = 0; rep < 3 && st == CT_OK; ++rep) {
                CT_CUDA(cudaMemcpyAsync(ct->d_domScratch, trial->data(), trial->size() * sizeof(uint32_t),
                                        cudaMemcpyHostToDevice, ct->stream));
                CT_CUDA(cudaStreamSynchronize(ct->stream));
                const auto t0 = std::chrono::steady_clock::now();
                const int r = ct_table_propagate_on(ct, ct->d_domScratch, ct->dev.varLD, ct->ld.data(), nullptr);
                const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (r < 0) st = r;
                tmin = std::min(tmin, dt);
                if (st == CT_OK && (st = ct_restore(ct, L)) == CT_OK) st = ct_save(ct, &L);
            }
            score += tmin;
        }
        if (st != CT_OK) break;
        if (score < best) {
            best = score;
            bestVar = c.first;
            bestGrid = c.second;
        }
    }
    const int rs = ct_restore(ct, L);
    ct->variant = st == CT_OK ? bestVar : saveVar;
    ct->grid = st == CT_OK ? bestGrid : saveGrid;
    ct->profile = saveProfile;
    ct->prof = ct_profile{};
    ct->autotuned = st == CT_OK;
    return st != CT_OK ? st : rs;
}

}  // namespace

namespace {
int create_impl(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples, int64_t t,
                const ct_options* opt, void* cuda_stream, ct_table** out, bool negative);
}  // namespace

extern "C" int ct_debug_guard_buffers(int on) {
    std::lock_guard<std::mutex> lk(g_bufMu);
    g_guardNew = on != 0;
    return CT_OK;
}

extern "C" int ct_debug_fail_alloc(int n) {
    std::lock_guard<std::mutex> lk(g_bufMu);
    g_failAfter = n < 0 ? -1 : n;
    return CT_OK;
}

extern "C" int ct_debug_device_bytes(int64_t* bytes_out) {
    if (!bytes_out) {
        ct_set_error("ct_debug_device_bytes: bytes_out is null");
        return CT_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_bufMu);
    *bytes_out = g_bufBytes;
    return CT_OK;
}

extern "C" int ct_debug_check_guards(ct_table* ct, int poke, int64_t* changed_out) {
    if (!ct || !changed_out || poke < 0 || poke > (int)kGuardBytes) {
        ct_set_error("ct_debug_check_guards: a table, changed_out, and 0 <= poke <= %d", (int)kGuardBytes);
        return CT_ERR_ARG;
    }
    if (ct->stream) CT_CUDA(cudaStreamSynchronize(ct->stream));
    std::vector<void*> bufs(ct->allocs.begin(), ct->allocs.end());
    if (!ct->trailInArena) {
        bufs.push_back(ct->dev.trailKey);
        bufs.push_back(ct->dev.trailOld);
    }
    if (!ct->levelsInArena) {
        bufs.push_back(ct->dev.levelSeg);
        bufs.push_back(ct->dev.levelDom);
    }
    std::vector<std::pair<char*, size_t>> guarded;
    {
        std::lock_guard<std::mutex> lk(g_bufMu);
        for (void* b : bufs) {
            const auto it = b ? g_bufs.find(b) : g_bufs.end();
            if (it != g_bufs.end() && it->second.guarded) guarded.emplace_back(static_cast<char*>(b), it->second.bytes);
        }
    }
    if (poke > 0 && !guarded.empty())
        CT_CUDA(cudaMemset(guarded[0].first - kGuardBytes, 0, (size_t)poke));  // from the host: no kernel writes it
    CT_CUDA(cudaDeviceSynchronize());
    int64_t changed = 0;
    std::vector<unsigned char> h(kGuardBytes);
    for (const auto& g : guarded) {
        for (int side = 0; side < 2; ++side) {
            const char* at = side == 0 ? g.first - kGuardBytes : g.first + g.second;
            CT_CUDA(cudaMemcpy(h.data(), at, kGuardBytes, cudaMemcpyDeviceToHost));
            for (unsigned char c : h) changed += c != kGuardFill;
        }
    }
    *changed_out = changed;
    return CT_OK;
}

extern "C" int ct_create(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples,
                         int64_t t, const ct_options* opt, void* cuda_stream, ct_table** out) {
    return create_impl(arity, dom_lo, dom_size, tuples, t, opt, cuda_stream, out, false);
}

extern "C" int ct_create_negative(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples,
                                  int64_t t, const ct_options* opt, void* cuda_stream, ct_table** out) {
    return create_impl(arity, dom_lo, dom_size, tuples, t, opt, cuda_stream, out, true);
}

int ct_table_is_negative(const ct_table* ct) { return ct->negative ? 1 : 0; }

namespace {
int create_impl(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples, int64_t t,
                const ct_options* opt, void* cuda_stream, ct_table** out, bool negative) {
    if (!out) {
        ct_set_error("ct_create: out is null");
        return CT_ERR_ARG;
    }
    *out = nullptr;
    if (arity < 1 || arity > kMaxArity || !dom_lo || !dom_size || t < 0 || (t > 0 && !tuples)) {
        ct_set_error("ct_create: invalid arity/domains/tuples (arity %d, t %lld)", arity, (long long)t);
        return CT_ERR_ARG;
    }
    for (int i = 0; i < arity; ++i) {
        if (dom_size[i] < 1 || dom_size[i] > kMaxDomSize) {
            ct_set_error("ct_create: dom_size[%d] = %d out of [1, %d]", i, dom_size[i], kMaxDomSize);
            return CT_ERR_ARG;
        }
    }
    if (negative && opt && opt->shard) {
        ct_set_error("ct_create_negative: negative tables cannot be shards");
        return CT_ERR_ARG;
    }
    ct_table* ct = new (std::nothrow) ct_table();
    if (!ct) return CT_ERR_OOM;
    ct->arity = arity;
    if (cuda_stream) {
        ct->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        const cudaError_t e = cudaStreamCreateWithFlags(&ct->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ct;
            return ct_cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        ct->ownStream = true;
    }
    const int st = build(ct, dom_lo, dom_size, tuples, t, opt, negative);
    if (st < 0) {
        free_table(ct);
        return st;
    }
    if (st == CT_OK && opt && opt->autotune && opt->grid_blocks <= 0) {
        const int at = autotune(ct);
        if (at < 0) {
            free_table(ct);
            return at;
        }
    }
    *out = ct;
    return st;
}
}  // namespace

extern "C" int ct_propagate(ct_table* ct, uint32_t* dom_bits, uint32_t* changed_vars) {
    if (!ct) {
        ct_set_error("ct_propagate: null handle");
        return CT_ERR_ARG;
    }
    return ct_table_propagate_on(ct, dom_bits, ct->dev.varLD, ct->ld.data(), changed_vars);
}

extern "C" int ct_arm_wait_timeout(ct_table* ct, uint32_t polls) {
    if (polls == 0) {
        ct_set_error("ct_arm_wait_timeout: polls must be positive");
        return CT_ERR_ARG;
    }
    if (!ct) return ct_noalloc_arm_wait_timeout(polls);
    ct->armPolls = polls;
    return CT_OK;
}

extern "C" int ct_propagate_host(ct_table* ct, uint32_t* dom_bits_host, uint32_t* changed_vars) {
    if (!ct || !dom_bits_host) {
        ct_set_error("ct_propagate_host: null argument");
        return CT_ERR_ARG;
    }
    if (ct->empty) return ct_table_propagate_on(ct, dom_bits_host, nullptr, nullptr, changed_vars);
    int st;
    if (ct->localPlan && ct->DW <= kParamDomWords && !ct->copyState) {
        // a few domain words: they go to the device with the launch itself
        st = ct_table_propagate_on(ct, nullptr, ct->dev.varLD, ct->ld.data(), changed_vars, dom_bits_host);
    } else {
        CT_CUDA(cudaMemcpyAsync(ct->d_domScratch, dom_bits_host, (size_t)ct->DW * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, ct->stream));
        st = ct_table_propagate_on(ct, ct->d_domScratch, ct->dev.varLD, ct->ld.data(), changed_vars);
    }
    if (st == CT_OK && ct->h_status[kSlotPruned] > 0) {
        // Only the variables that lost values differ from the input.
        const int32_t* h = ct->h_status;
        const uint32_t* outDom = reinterpret_cast<const uint32_t*>(h + kStatusHdr + ct->nChW);
        for (int i = 0; i < ct->arity; ++i) {
            if (!(((uint32_t)h[kStatusHdr + (i >> 5)] >> (i & 31)) & 1u)) continue;
            std::memcpy(dom_bits_host + ct->ld[i], outDom + ct->ld[i], (size_t)ct->nw[i] * sizeof(uint32_t));
        }
    }
    return st;
}

extern "C" int ct_save(ct_table* ct, int* level_out) {
    if (!ct) {
        ct_set_error("ct_save: null handle");
        return CT_ERR_ARG;
    }
    if (ct->failed) {
        ct_set_error("ct_save: the previous call failed; restore a level first");
        return CT_ERR_STATE;
    }
    const int L = (int)ct->levels.size();
    if (!ct->empty) {
        int st;
        if ((st = ensure_levels(ct, L + 1)) != CT_OK) return st;
    }
    // The snapshot itself is taken by the next propagation (or never, if the
    // level is restored before any propagation changed the state).
    ct->levels.push_back(ct_table::Level{ct->trailTop, ct->live, L});
    if (level_out) *level_out = L;
    return CT_OK;
}

extern "C" int ct_restore(ct_table* ct, int level) {
    if (!ct) {
        ct_set_error("ct_restore: null handle");
        return CT_ERR_ARG;
    }
    if (level < 0 || level >= (int)ct->levels.size()) {
        ct_set_error("ct_restore: level %d not in [0, %d)", level, (int)ct->levels.size());
        return CT_ERR_LEVEL;
    }
    if (ct->broken) {
        ct_set_error("ct_restore: the table is unusable after a device-side timeout");
        return CT_ERR_TIMEOUT;
    }
    const int mark = ct->levels[level].mark;
    if (!ct->empty && level < ct->pendingFrom) {
        CT_CUDA(launch_restore(ct->dev, ct->levels[level].snap, mark, ct->trailTop, -1, ct->stream));
        ct->trailTop = mark;
        if (ct->copyState && ct->h_curr) {
            const int st = fetch_host_curr(ct);
            if (st != CT_OK) return st;
        }
    }
    // A level saved after the last propagation still equals the current state.
    ct->failed = false;
    ct->live = ct->levels[level].live;
    ct->levels.resize(level);
    ct->pendingFrom = std::min(ct->pendingFrom, level);
    return CT_OK;
}

extern "C" int ct_get_currtable(ct_table* ct, uint32_t* words_host, int64_t* nonzero_words_out) {
    if (!ct) {
        ct_set_error("ct_get_currtable: null handle");
        return CT_ERR_ARG;
    }
    if (ct->empty) {
        if (nonzero_words_out) *nonzero_words_out = 0;
        return CT_OK;
    }
    std::vector<uint32_t> buf((size_t)ct->W4 * 4);
    CT_CUDA(cudaMemcpyAsync(buf.data(), ct->dev.curr, buf.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            ct->stream));
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    int64_t nz = 0;
    for (int64_t w = 0; w < ct->W; ++w) nz += buf[(size_t)w] != 0u;
    if (words_host) std::memcpy(words_host, buf.data(), (size_t)ct->W * sizeof(uint32_t));
    if (nonzero_words_out) *nonzero_words_out = nz;
    return CT_OK;
}

extern "C" int ct_get_support_row(ct_table* ct, int row, uint32_t* words_host) {
    if (!ct || !words_host || row < 0 || row >= ct->R) {
        ct_set_error("ct_get_support_row: bad argument");
        return CT_ERR_ARG;
    }
    if (ct->empty) return CT_OK;
    CT_CUDA(cudaMemcpyAsync(words_host, ct->dev.sup + (size_t)row * ct->W4, (size_t)ct->W * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, ct->stream));
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    return CT_OK;
}

extern "C" int ct_get_index(ct_table* ct, int32_t* index_host, int64_t* count_out) {
    if (!ct) {
        ct_set_error("ct_get_index: null handle");
        return CT_ERR_ARG;
    }
    if (ct->empty) {
        if (count_out) *count_out = 0;
        return CT_OK;
    }
    std::vector<uint32_t> mask(ct->nseg);
    CT_CUDA(cudaMemcpyAsync(mask.data(), ct->dev.segMask, mask.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            ct->stream));
    CT_CUDA(cudaStreamSynchronize(ct->stream));
    int64_t n = 0;
    for (int s = 0; s < ct->nseg; ++s) {
        for (int j = 0; j < 32; ++j) {
            if (!((mask[s] >> j) & 1u)) continue;
            if (index_host) index_host[n] = s * 32 + j;
            ++n;
        }
    }
    if (count_out) *count_out = n;
    return CT_OK;
}

extern "C" int ct_get_info(ct_table* ct, ct_table_info* info) {
    if (!ct || !info) {
        ct_set_error("ct_get_info: null argument");
        return CT_ERR_ARG;
    }
    ct_table_info r{};
    r.arity = ct->arity;
    r.rows = ct->R;
    r.tuples = ct->t;
    r.words = ct->W;
    r.chunks = ct->W4;
    r.segments = ct->nseg;
    r.seg_capacity = ct->S;
    r.trail_size = ct->trailTop;
    r.depth = (int)ct->levels.size();
    r.local_plan = ct->localPlan ? 1 : 0;
    r.grid_blocks = ct->grid;
    r.short_tuples = (int32_t)std::min<int64_t>(ct->shortTuples, 0x7fffffff);
    r.loads_in_flight = (ct->variant & 2) ? 8 : 16;
    r.autotuned = ct->autotuned ? 1 : 0;
    r.device_bytes = ct->deviceBytes;
    int64_t live = 0;
    const int st = ct_get_index(ct, nullptr, &live);
    if (st != CT_OK) return st;
    r.live_chunks = live;
    *info = r;
    return CT_OK;
}

extern "C" int ct_get_call_stats(ct_table* ct, ct_call_stats* stats) {
    if (!ct || !stats) {
        ct_set_error("ct_get_call_stats: null argument");
        return CT_ERR_ARG;
    }
    *stats = ct->last;
    return CT_OK;
}

extern "C" int ct_get_profile(ct_table* ct, ct_profile* prof) {
    if (!ct || !prof) {
        ct_set_error("ct_get_profile: null argument");
        return CT_ERR_ARG;
    }
    const int st = drain_events(ct);
    if (st != CT_OK) return st;
    *prof = ct->prof;
    return CT_OK;
}

extern "C" int ct_set_profile(ct_table* ct, int on) {
    if (!ct) {
        ct_set_error("ct_set_profile: null handle");
        return CT_ERR_ARG;
    }
    if (on && ct->ev.empty()) {
        const int st = create_events(ct);
        if (st != CT_OK) return st;
    }
    if (!on) {
        const int st = drain_events(ct);
        if (st != CT_OK) return st;
    }
    ct->profile = on != 0;
    return CT_OK;
}

extern "C" int ct_reset_profile(ct_table* ct) {
    if (!ct) return CT_ERR_ARG;
    const int st = drain_events(ct);
    ct->prof = ct_profile{};
    return st;
}

extern "C" int ct_destroy(ct_table* ct) {
    free_table(ct);
    return CT_OK;
}
