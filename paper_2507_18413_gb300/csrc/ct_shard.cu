// ct_shard.cu -- one table split into K word-range shards on one device: the
// data-parallel form of a single table's propagation. Each shard holds a
// contiguous range of the retained tuples (whole 128-tuple chunks), runs
// updateTable on its own currTable words, and reports the values its own valid
// tuples support; the supported sets are OR-combined (the all-reduce of the
// split, here one small kernel) into the new domains. GAC of the whole table
// is the union over the shards, since a value is supported iff some valid
// tuple, in whichever shard, carries it (Sec. 2); the table fails iff every
// shard's currTable is empty, i.e. iff a combined domain is empty.
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "ct.h"
#include "ct_internal.cuh"

namespace {

constexpr int64_t kChunkTuples = 128;  // tuples per 128-bit currTable chunk

// dom[q] := OR over the K shard outputs; per-variable changed bits and the
// number of emptied variables go to the mapped result block (one CTA; the
// changed bits are gathered in shared memory, nChW words).
__global__ void ct_shard_or_kernel(uint32_t* __restrict__ dom, const uint32_t* __restrict__ scratch, int K, int DW,
                                   const int32_t* __restrict__ varOff, const int32_t* __restrict__ varNW, int arity,
                                   int32_t* __restrict__ res) {
    extern __shared__ unsigned chgBits[];
    __shared__ int empties;
    const int nChW = (arity + 31) / 32;
    for (int q = threadIdx.x; q < nChW; q += blockDim.x) chgBits[q] = 0u;
    if (threadIdx.x == 0) empties = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < arity; i += blockDim.x) {
        bool any = false, chg = false;
        for (int q = varOff[i]; q < varOff[i] + varNW[i]; ++q) {
            uint32_t v = 0u;
            for (int k = 0; k < K; ++k) v |= scratch[(size_t)k * DW + q];
            chg |= v != dom[q];
            any |= v != 0u;
            dom[q] = v;
        }
        if (!any) atomicAdd(&empties, 1);
        if (chg) atomicOr(&chgBits[i >> 5], 1u << (i & 31));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nChW; q += blockDim.x) res[1 + q] = (int32_t)chgBits[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence_system();
        res[0] = empties;
    }
}

}  // namespace

struct ct_sharded {
    int K = 0, arity = 0, DW = 0, nChW = 0;
    std::vector<ct_table*> shards;
    std::vector<int64_t> bounds;  // K + 1 retained-tuple positions
    uint32_t* d_scratch = nullptr;  // [K][DW] per-shard domains
    int32_t* d_layout = nullptr;    // [arity] word offsets, then [arity] word counts
    int32_t* h_res = nullptr;       // mapped: [0] emptied variables, then changed bits
    int32_t* d_res = nullptr;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    bool ownStream = false;
};

extern "C" int ct_shard_bounds(int64_t t, int K, int64_t* bounds_out) {
    if (t < 1 || K < 1 || !bounds_out) {
        ct_set_error("ct_shard_bounds: t >= 1, K >= 1 and an output array are needed");
        return CT_ERR_ARG;
    }
    const int64_t chunks = (t + kChunkTuples - 1) / kChunkTuples;
    if (K > chunks) {
        ct_set_error("ct_shard_bounds: %d shards for %lld chunks of 128 tuples", K, (long long)chunks);
        return CT_ERR_ARG;
    }
    for (int k = 0; k <= K; ++k) {
        const int64_t c = chunks * k / K;
        bounds_out[k] = c * kChunkTuples < t ? c * kChunkTuples : t;
    }
    return CT_OK;
}

extern "C" int ct_sharded_destroy(ct_sharded* sh) {
    if (!sh) return CT_OK;
    for (ct_table* t : sh->shards) ct_destroy(t);
    if (sh->d_scratch) cudaFree(sh->d_scratch);
    if (sh->d_layout) cudaFree(sh->d_layout);
    if (sh->h_res) cudaFreeHost(sh->h_res);
    if (sh->ownStream && sh->stream) cudaStreamDestroy(sh->stream);
    cudaGetLastError();
    delete sh;
    return CT_OK;
}

extern "C" int ct_sharded_create(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples,
                                 int64_t t, int K, const ct_options* opt, void* cuda_stream, ct_sharded** out) {
    if (!out) {
        ct_set_error("ct_sharded_create: out is null");
        return CT_ERR_ARG;
    }
    *out = nullptr;
    if (arity < 1 || !dom_lo || !dom_size || t < 0 || (t > 0 && !tuples) || K < 1) {
        ct_set_error("ct_sharded_create: invalid arguments (arity %d, t %lld, K %d)", arity, (long long)t, K);
        return CT_ERR_ARG;
    }
    for (int i = 0; i < arity; ++i) {
        if (dom_size[i] < 1) {
            ct_set_error("ct_sharded_create: dom_size[%d] = %d", i, dom_size[i]);
            return CT_ERR_ARG;
        }
    }
    // Retained tuples in input order (the positions of the whole table).
    std::vector<int32_t> kept;
    kept.reserve((size_t)t * arity);
    int64_t n = 0;
    for (int64_t j = 0; j < t; ++j) {
        const int32_t* tu = tuples + j * arity;
        bool ok = true;
        for (int i = 0; i < arity && ok; ++i)
            ok = tu[i] == CT_STAR || ((int64_t)tu[i] >= dom_lo[i] && (int64_t)tu[i] - dom_lo[i] < dom_size[i]);
        if (ok) {
            kept.insert(kept.end(), tu, tu + arity);
            ++n;
        }
    }
    if (n == 0) {
        ct_set_error("ct_sharded_create: no tuple inside the domains");
        return CT_INFEASIBLE;
    }
    ct_sharded* sh = new (std::nothrow) ct_sharded();
    if (!sh) return CT_ERR_OOM;
    sh->K = K;
    sh->arity = arity;
    sh->t = n;
    sh->nChW = (arity + 31) / 32;
    sh->bounds.resize((size_t)K + 1);
    int st = ct_shard_bounds(n, K, sh->bounds.data());
    if (st != CT_OK) {
        delete sh;
        return st;
    }
    if (cuda_stream) {
        sh->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        const cudaError_t e = cudaStreamCreateWithFlags(&sh->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete sh;
            return ct_cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        sh->ownStream = true;
    }
    ct_options o{};
    if (opt) o = *opt;
    o.shard = 1;
    for (int k = 0; k < K; ++k) {
        ct_table* tab = nullptr;
        const int64_t b0 = sh->bounds[k], b1 = sh->bounds[k + 1];
        st = ct_create(arity, dom_lo, dom_size, kept.data() + b0 * arity, b1 - b0, &o, sh->stream, &tab);
        if (st != CT_OK) {
            if (tab) ct_destroy(tab);
            ct_sharded_destroy(sh);
            return st < 0 ? st : CT_ERR_STATE;
        }
        sh->shards.push_back(tab);
    }
    std::vector<int32_t> layout(2 * (size_t)arity);
    int DW = 0;
    for (int i = 0; i < arity; ++i) {
        layout[i] = DW;
        layout[arity + i] = (dom_size[i] + 31) / 32;
        DW += layout[arity + i];
    }
    sh->DW = DW;
    cudaError_t e = cudaMalloc(&sh->d_scratch, (size_t)K * DW * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&sh->d_layout, layout.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sh->d_layout, layout.data(), layout.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            sh->stream);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void**)&sh->h_res, (1 + (size_t)sh->nChW) * sizeof(int32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sh->d_res, sh->h_res, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sh->stream);
    if (e != cudaSuccess) {
        st = ct_cuda_fail(e, "ct_sharded_create");
        ct_sharded_destroy(sh);
        return st;
    }
    *out = sh;
    return CT_OK;
}

extern "C" int ct_sharded_propagate(ct_sharded* sh, uint32_t* dom_bits, uint32_t* changed_vars) {
    if (!sh || !dom_bits) {
        ct_set_error("ct_sharded_propagate: null argument");
        return CT_ERR_ARG;
    }
    const size_t bytes = (size_t)sh->DW * sizeof(uint32_t);
    for (int k = 0; k < sh->K; ++k) {
        uint32_t* d = sh->d_scratch + (size_t)k * sh->DW;
        CT_CUDA(cudaMemcpyAsync(d, dom_bits, bytes, cudaMemcpyDeviceToDevice, sh->stream));
        const int st = ct_propagate(sh->shards[k], d, nullptr);
        if (st != CT_OK) {
            if (st == CT_INFEASIBLE) ct_set_error("ct_sharded_propagate: an input domain is empty");
            return st < 0 ? st : CT_ERR_STATE;
        }
    }
    std::memset(sh->h_res, 0, (1 + (size_t)sh->nChW) * sizeof(int32_t));
    sh->h_res[0] = -1;
    ct_shard_or_kernel<<<1, 256, (size_t)sh->nChW * sizeof(unsigned), sh->stream>>>(
        dom_bits, sh->d_scratch, sh->K, sh->DW, sh->d_layout, sh->d_layout + sh->arity, sh->arity, sh->d_res);
    CT_CUDA(cudaGetLastError());
    CT_CUDA(cudaStreamSynchronize(sh->stream));
    if (changed_vars) std::memcpy(changed_vars, sh->h_res + 1, (size_t)sh->nChW * sizeof(uint32_t));
    return sh->h_res[0] > 0 ? CT_INFEASIBLE : CT_OK;
}

extern "C" int ct_sharded_save(ct_sharded* sh, int* level_out) {
    if (!sh) {
        ct_set_error("ct_sharded_save: null handle");
        return CT_ERR_ARG;
    }
    int level = 0;
    for (ct_table* t : sh->shards) {
        const int st = ct_save(t, &level);
        if (st != CT_OK) return st;
    }
    if (level_out) *level_out = level;
    return CT_OK;
}

extern "C" int ct_sharded_restore(ct_sharded* sh, int level) {
    if (!sh) {
        ct_set_error("ct_sharded_restore: null handle");
        return CT_ERR_ARG;
    }
    for (ct_table* t : sh->shards) {
        const int st = ct_restore(t, level);
        if (st != CT_OK) return st;
    }
    return CT_OK;
}

extern "C" int ct_sharded_get_currtable(ct_sharded* sh, uint32_t* words_host, int64_t* nonzero_words_out) {
    if (!sh) {
        ct_set_error("ct_sharded_get_currtable: null handle");
        return CT_ERR_ARG;
    }
    int64_t nz = 0;
    for (int k = 0; k < sh->K; ++k) {
        int64_t z = 0;
        // shard k starts at a multiple of 128 tuples: word bounds[k] / 32
        const int st = ct_get_currtable(sh->shards[k], words_host ? words_host + sh->bounds[k] / 32 : nullptr, &z);
        if (st != CT_OK) return st;
        nz += z;
    }
    if (nonzero_words_out) *nonzero_words_out = nz;
    return CT_OK;
}

extern "C" int ct_sharded_get_shard(ct_sharded* sh, int k, ct_table** table_out) {
    if (!sh || !table_out || k < 0 || k >= sh->K) {
        ct_set_error("ct_sharded_get_shard: null handle or shard %d not in [0, K)", k);
        return CT_ERR_ARG;
    }
    *table_out = sh->shards[k];
    return CT_OK;
}
