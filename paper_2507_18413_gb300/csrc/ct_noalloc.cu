// ct_noalloc.cu -- one propagation on caller-owned buffers, with no allocation.
//
// Some callers cannot allocate device memory at the time they propagate: code
// that runs under a memory pool or arena owned by another framework, code
// whose allocations must all happen at start-up (real-time or long-running
// services that forbid allocation on the hot path), or code that must not
// trigger the implicit device synchronisation of cudaMalloc/cudaFree. For
// them ct_propagate_noalloc runs the same propagation kernel as ct_propagate
// on buffers the caller owns (supports, currTable, domains, last domains)
// and keeps its scratch (the update plan, the hard-value list, counters, the
// grid barrier, the status block) in the file-scope array below, which every
// GPU that loads the library holds until the process exits. It neither
// allocates nor frees anything: no cudaMalloc, no cudaFree, no pinned host
// memory, no allocating library call.
//
// Limits of this entry point: at most kNaMaxArity scope variables, at most
// kNaMaxRows supports rows (sum of the domain sizes) and kNaMaxChunks 128-bit
// chunks of currTable (8,388,608 tuples). Backtracking is the caller's
// business (it keeps copies of the buffers it wants to return to).
#include <atomic>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "ct_internal.cuh"

using namespace ctk;

namespace {

constexpr int kNaMaxArity = kParamArity;  // 16
constexpr int kNaMaxRows = 1024;
constexpr int kNaMaxChunks = 65536;
constexpr int kNaMaxSeg = kNaMaxChunks / 32;
constexpr int kNaMaxDW = 64;  // sum of ceil(dom_size / 32) is below this when the rows fit
constexpr int kNaMaxDevices = 64;
constexpr int32_t kNaPending = 0x7f7f7f7f;  // status word before the kernel publishes

struct NaScratch {
    Ctrl ctrl;
    int32_t status[kStatusHdr + 1 + kNaMaxDW];
    uint32_t segMask[kNaMaxSeg];
    int32_t codes[kNaMaxRows];
    int32_t hardRow[kNaMaxRows];
    int32_t foundChunk[kNaMaxRows];
    int32_t residue[kNaMaxRows];
    int32_t rowVar[kNaMaxRows];
    int32_t varSup[kNaMaxArity];
    int32_t planK[kNaMaxArity];
    int32_t planRowOff[kNaMaxArity];
};

// The scratch of every ct_propagate_noalloc call on a device (about 32 KB).
static __device__ __align__(256) unsigned char g_ct_noalloc_scratch[sizeof(NaScratch)];

// Per-call initialisation of the scratch: everything it needs is in the
// kernel parameters, so no host buffer is read after the launch.
struct NaInit {
    int32_t rowVar[kNaMaxRows];  // scope position of each supports row
    int32_t R;
    int32_t nseg;
    int32_t W4;                  // 128-bit chunks of currTable
    uint32_t barCount;           // initial grid-barrier count (0; the timeout test hook sets it 2^30 behind)
    const uint4* curr;           // the caller's currTable
};

// The non-zero index of the caller's currTable is rebuilt from its chunks
// (one warp ballot per 32-chunk segment), so dead chunks left by earlier calls
// are neither read by updateTable nor scanned by filterDomains.
__global__ void ct_noalloc_init_kernel(const __grid_constant__ NaInit p) {
    NaScratch* S = reinterpret_cast<NaScratch*>(g_ct_noalloc_scratch);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    int32_t* c = reinterpret_cast<int32_t*>(&S->ctrl);
    // one writer per word: the barrier count starts at p.barCount, the rest at 0
    constexpr int kBarWord = (int)(offsetof(Ctrl, bar_count) / sizeof(int32_t));
    for (int q = tid; q < (int)(sizeof(Ctrl) / sizeof(int32_t)); q += nth) c[q] = q == kBarWord ? (int32_t)p.barCount : 0;
    for (int q = tid; q < p.R; q += nth) {
        S->residue[q] = 0;
        S->rowVar[q] = p.rowVar[q];
    }
    const int lane = threadIdx.x & 31;
    for (int seg0 = (tid >> 5) << 5; seg0 < p.nseg * 32; seg0 += nth) {
        const int w = seg0 + lane;  // chunk; seg0 is a multiple of 32
        bool live = false;
        if (w < p.W4) {
            const uint4 v = p.curr[w];
            live = (v.x | v.y | v.z | v.w) != 0u;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, live);
        if (lane == 0) S->segMask[seg0 >> 5] = m;
    }
    if (tid == 0) {
        S->status[kSlotStatus] = kNaPending;
    }
}

std::atomic<uint32_t> g_na_arm{0};  // test hook: polls of the next call's barrier waits (0: off)

struct NaDevice {
    NaScratch* scratch = nullptr;  // device address of g_ct_noalloc_scratch
    int maxCo[4] = {0, 0, 0, 0};   // co-resident CTAs of each kernel variant
};

std::mutex g_na_mutex;
NaDevice g_na[kNaMaxDevices];

// Once per device, with that device current: the device address of the
// scratch array (in host code its name is only a stand-in for the symbol) and
// the residency of the kernel variants.
int na_setup(int dev, NaDevice** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaDevice& d = g_na[dev];
    if (!d.scratch) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ct_noalloc_scratch);
        if (e != cudaSuccess) return ct_cuda_fail(e, "cudaGetSymbolAddress(g_ct_noalloc_scratch)");
        d.maxCo[1] = max_coresident_blocks(1);
        d.maxCo[3] = max_coresident_blocks(3);
        if (d.maxCo[1] <= 0 || d.maxCo[3] <= 0) {
            ct_set_error("ct_propagate_noalloc: the propagation kernel cannot be made resident on this device");
            return CT_ERR_CUDA;
        }
        d.scratch = static_cast<NaScratch*>(p);
    }
    *out = &d;
    return CT_OK;
}

}  // namespace

int ct_noalloc_arm_wait_timeout(uint32_t polls) {
    g_na_arm.store(polls);
    return CT_OK;
}

extern "C" int ct_propagate_noalloc(int arity, const int32_t* dom_size, int64_t t, const uint32_t* supports,
                                    uint32_t* curr_table, uint32_t* dom_bits, uint32_t* last_dom_bits,
                                    uint32_t* changed_vars, void* cuda_stream) {
    if (arity < 1 || arity > kNaMaxArity || !dom_size || t < 1 || !supports || !curr_table || !dom_bits ||
        !last_dom_bits) {
        ct_set_error("ct_propagate_noalloc: arity must be in [1, %d], t >= 1 and every buffer given", kNaMaxArity);
        return CT_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(supports) | reinterpret_cast<uintptr_t>(curr_table)) & 15u) {
        ct_set_error("ct_propagate_noalloc: supports and curr_table must be 16-byte aligned");
        return CT_ERR_ARG;
    }
    int nw[kNaMaxArity], ld[kNaMaxArity], row0[kNaMaxArity];
    int R = 0, DW = 0;
    for (int i = 0; i < arity; ++i) {
        if (dom_size[i] < 1 || dom_size[i] > kNaMaxRows) {
            ct_set_error("ct_propagate_noalloc: dom_size[%d] = %d out of [1, %d]", i, dom_size[i], kNaMaxRows);
            return CT_ERR_ARG;
        }
        nw[i] = (dom_size[i] + 31) / 32;
        ld[i] = DW;
        row0[i] = R;
        DW += nw[i];
        R += dom_size[i];
    }
    const int64_t W4 = ((t + 31) / 32 + 3) / 4;
    if (R > kNaMaxRows || W4 > kNaMaxChunks || DW > kNaMaxDW) {
        ct_set_error("ct_propagate_noalloc: %d supports rows and %lld chunks exceed the limits (%d rows, %d chunks)",
                     R, (long long)W4, kNaMaxRows, kNaMaxChunks);
        return CT_ERR_ARG;
    }
    int dev = 0;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        ct_set_error("ct_propagate_noalloc: device ordinal %d beyond %d", dev, kNaMaxDevices);
        return CT_ERR_ARG;
    }
    NaDevice* nd = nullptr;
    int st = na_setup(dev, &nd);
    if (st != CT_OK) return st;
    NaScratch* S = nd->scratch;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    const int nseg = (int)((W4 + 31) / 32);
    TableDev T{};
    T.sup = reinterpret_cast<const uint4*>(supports);
    T.supDelta = T.sup;
    T.curr = reinterpret_cast<uint4*>(curr_table);
    T.segMask = S->segMask;
    T.residue = S->residue;
    T.lastDom = last_dom_bits;
    T.ctrl = &S->ctrl;
    T.codes = S->codes;
    T.planK = S->planK;
    T.planRowOff = S->planRowOff;
    T.varSup = S->varSup;
    T.other = nullptr;  // positive tables only
    T.hardRow = S->hardRow;
    T.foundChunk = S->foundChunk;
    T.rowVar = S->rowVar;
    T.statusBlk = S->status;
    T.arity = arity;
    T.R = R;
    T.W4 = (int32_t)W4;
    T.nseg = nseg;
    T.S = 32;
    T.DW = DW;
    T.nChangedWords = 1;
    T.useResidues = 1;
    for (int i = 0; i < arity; ++i) {
        T.pNW[i] = nw[i];
        T.pLD[i] = ld[i];
        T.pRow0[i] = row0[i];
    }

    // The array keeps the previous call's contents: clear what must start at
    // zero (counters and barrier, residues), rebuild the
    // non-zero index from the caller's currTable, reload the row -> variable
    // map, reset the status word.
    NaInit init;
    for (int i = 0; i < arity; ++i)
        for (int a = 0; a < dom_size[i]; ++a) init.rowVar[row0[i] + a] = i;
    init.R = R;
    init.nseg = nseg;
    init.W4 = (int32_t)W4;
    init.curr = T.curr;
    const uint32_t armed = g_na_arm.exchange(0u);
    init.barCount = armed ? 0xC0000000u : 0u;
    ct_noalloc_init_kernel<<<8, 256, 0, s>>>(init);
    CT_CUDA(cudaGetLastError());

    CallParams P{};
    P.mark = -1;  // no backtrack levels: nothing is trailed
    P.snapFrom = 0;
    P.snapTo = 0;
    P.prevLive = (int32_t)W4;
    P.spinLimit = armed ? armed : kBarrierSpinLimit;
    P.maxSplit = 1;
    for (int i = 0; i < arity; ++i) P.domOff[i] = ld[i];
    const int variant = nseg > nd->maxCo[1] * kWarps ? 3 : 1;
    int grid = (nseg + kWarps - 1) / kWarps;
    grid = grid > (R + 2 * kWarps - 1) / (2 * kWarps) ? grid : (R + 2 * kWarps - 1) / (2 * kWarps);
    if (grid > nd->maxCo[variant]) grid = nd->maxCo[variant];
    if (grid < 1) grid = 1;
    CT_CUDA(launch_propagate(T, variant, grid, dom_bits, nullptr, P, s));

    int32_t head[kStatusHdr + 1];
    CT_CUDA(cudaMemcpyAsync(head, S->status, sizeof(head), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    const int status = head[kSlotStatus];
    if (status == kNaPending) {
        ct_set_error("ct_propagate_noalloc: the kernel did not publish a result (a device-side wait ran out)");
        return CT_ERR_TIMEOUT;
    }
    if (status == CT_ERR_STATE) ct_set_error("ct_propagate_noalloc: a domain grew since the last call");
    if (changed_vars) changed_vars[0] = (status == CT_OK && head[kSlotPruned] > 0) ? (uint32_t)head[kStatusHdr] : 0u;
    return status;
}
