// ct_learn.cu -- the learned branching order: per-variable features of a
// network's state, and the 8 -> 64 -> 64 -> 1 scoring network with its
// training (not in the paper, whose solver branches first-fail; Sec. 4).
//
// Features (kNF = 8 per variable, zero for |D(x)| < 2). With s = |D(x)|, d0
// the initial size, deg(x) the tables holding x (degmax the largest, >= 1),
// smax the largest |D| among the unfixed variables of the same node, and for
// every table c holding x with live_c > 0 valid tuples (tuples whose every
// value is in its current domain: the live bits of currTable),
// p_c(a) = |{valid tuples of c with x = a}| / live_c = popcount(supports[x,a]
// AND currTable) / popcount(currTable):
//   f0 = s / d0, f1 = log2(s) / 8, f2 = deg / degmax,
//   f3 = mean_c s * min_a p_c(a), f4 = mean_c max_a p_c(a),
//   f5 = mean_c (-sum_a p_c(a) log2 p_c(a)) / log2(s),
//   f6 = mean_c log2(1 + live_c) / 32, f7 = s / smax.
// The counts are integers (one warp per (table, segment), lane per chunk);
// the aggregation runs in double and is stored as float.
//
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), out = W3 . h2 + b3,
// float32, weights flat as W1[64][8], b1, W2[64][64], b2, W3[64], b3.
// Training: loss sum (out - y)^2 / (2B) per batch, Adam (Kingma and Ba, 2015;
// beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected), one CTA that keeps the
// weights, both moments and the batch's activations in shared memory and
// walks the given epoch orders in consecutive batches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ct_learn.cuh"

using namespace ctk;

struct ct_mlp {
    float* d_w = nullptr;  // [kNW]
    float* d_m = nullptr;  // Adam first moment
    float* d_v = nullptr;  // Adam second moment
    int64_t t = 0;         // Adam steps taken
    cudaStream_t stream = nullptr;
    bool ownStream = false;
};

namespace {

struct FeatArgs {
    const TableDev* tabs;
    const uint32_t* dom;
    const uint8_t* nodeActive;
    const int32_t* rowBase;
    const int32_t* unitBase;
    const int32_t* scopeBase;
    const int32_t* scopeOff;
    const int32_t* adjBase;
    const int2* adj;
    const int32_t* varOff;
    const int32_t* varNW;
    const int32_t* varD0;
    const int32_t* deg;
    uint32_t* counts;
    uint32_t* live;
    float* feat;
    int32_t nt, nv, T, V, degmax, totalUnits;
};

__device__ __forceinline__ uint32_t popc4(const uint4& v) {
    return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Valid tuples per supports row and per table: one warp per (table, segment,
// scope variable, domain word) unit, lane l holding live chunk 32 * segment +
// l. Only the rows of the word's present values are read, none for a fixed
// variable (its features are zero), eight row loads in flight; the unit of the
// first word of the first scope variable also counts the segment's valid
// tuples.
__global__ void ct_counts_kernel(const FeatArgs A) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int u = gwarp; u < A.totalUnits; u += nwarps) {
        int lo = 0, hi = A.nt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&A.unitBase[mid]) <= u) lo = mid;
            else hi = mid - 1;
        }
        const int t = lo;
        if (A.nodeActive && !A.nodeActive[t / A.T]) continue;
        const TableDev& T = A.tabs[t];
        const int s0 = __ldg(&A.scopeBase[t]);
        const int ar = __ldg(&A.scopeBase[t + 1]) - s0;
        int sw = 0;
        for (int k = 0; k < ar; ++k) sw += __ldg(&T.varNW[k]);
        const int local = u - __ldg(&A.unitBase[t]);
        const int seg = local / sw;
        int i = 0, q = local - seg * sw;
        while (i < ar && q >= __ldg(&T.varNW[i])) q -= __ldg(&T.varNW[i++]);
        if (i >= ar) continue;
        const uint32_t mask = T.segMask[seg];
        if (mask == 0u) continue;
        const int w = seg * 32 + lane;
        const bool act = (mask >> lane) & 1u;
        const uint4 cur = act ? T.curr[w] : make_uint4(0u, 0u, 0u, 0u);
        if (i == 0 && q == 0) {
            const uint32_t lv = warp_sum(popc4(cur));
            if (lane == 0 && lv) atomicAdd(&A.live[t], lv);
        }
        const uint32_t* dv = A.dom + __ldg(&A.scopeOff[s0 + i]);
        const int nw = __ldg(&T.varNW[i]);
        uint32_t sz = 0;
        for (int k = lane; k < nw; k += 32) sz += __popc(dv[k]);
        if (warp_sum(sz) < 2u) continue;
        const int row0 = __ldg(&T.varRow0[i]);
        const int base = __ldg(&A.rowBase[t]) + row0;
        const size_t W4 = (size_t)T.W4;
        const uint4* sp = T.sup + (size_t)row0 * W4 + w;
        {
            uint32_t bits = dv[q];
            while (bits) {
                int a[8];
                uint32_t n[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    a[j] = bits ? 32 * q + __ffs(bits) - 1 : -1;
                    bits &= bits - 1u;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    n[j] = 0u;
                    if (a[j] >= 0 && act) {
                        const uint4 s = __ldg(sp + (size_t)a[j] * W4);
                        n[j] = popc4(make_uint4(s.x & cur.x, s.y & cur.y, s.z & cur.z, s.w & cur.w));
                    }
                }
                // sums of the eight rows over the warp: three halving exchanges
                // leave lane l one row (4 b4 + 2 b3 + b2 of l), two more add it up
                const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
                uint32_t m4[4], m2[2];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    m4[k] = (h4 ? n[k + 4] : n[k]) + __shfl_xor_sync(0xffffffffu, h4 ? n[k] : n[k + 4], 16);
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    m2[k] = (h3 ? m4[k + 2] : m4[k]) + __shfl_xor_sync(0xffffffffu, h3 ? m4[k] : m4[k + 2], 8);
                uint32_t v = (h2 ? m2[1] : m2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? m2[0] : m2[1], 4);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                const int jr = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
                int ar = a[0];
#pragma unroll
                for (int j = 1; j < 8; ++j) ar = jr == j ? a[j] : ar;
                if ((lane & 3) == 0 && ar >= 0 && v) atomicAdd(&A.counts[base + ar], v);
            }
        }
    }
}

// Features of a node's variables: `perNode` CTAs per node, one warp per
// variable, lane l holding the values 32 q + l. Every CTA first takes the
// node's largest unfixed domain. Minimum and maximum counts are taken on the
// integers; the rest is float: a lane sums the entropy terms of its values
// (d / 32 of a domain of d values) before the warp reduction, a relative error
// of a few 1e-7 up to about a thousand values.
__global__ void ct_features_kernel(const FeatArgs A, int perNode) {
    const int node = blockIdx.x / perNode;
    if (A.nodeActive && !A.nodeActive[node]) return;
    __shared__ int red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int firstVar = (blockIdx.x - node * perNode) * nwarp;
    int mx = 0;
    for (int lx = tid; lx < A.V; lx += blockDim.x) {
        const int v = node * A.V + lx;
        int s = 0;
        for (int q = 0; q < A.varNW[v]; ++q) s += __popc(A.dom[A.varOff[v] + q]);
        if (s >= 2 && s > mx) mx = s;
    }
    mx = (int)warp_max((uint32_t)mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    int smax = 0;
    for (int k = 0; k < nwarp; ++k) smax = max(smax, red[k]);
    for (int lx = firstVar + warp; lx < A.V && lx < firstVar + nwarp; lx += nwarp) {
        const int v = node * A.V + lx;
        float* f = A.feat + (size_t)v * kNF;
        const uint32_t* d = A.dom + A.varOff[v];
        const int nw = A.varNW[v];
        uint32_t su = 0;
        for (int q = lane; q < nw; q += 32) su += __popc(d[q]);
        const int s = (int)warp_sum(su);
        if (s < 2) {
            if (lane < kNF) f[lane] = 0.0f;
            continue;
        }
        float bal = 0.0f, top = 0.0f, ent = 0.0f, liv = 0.0f;
        int cnt = 0;
        const float ls = log2f((float)s);
        for (int j = A.adjBase[v]; j < A.adjBase[v + 1]; ++j) {
            const int2 e = A.adj[j];
            const uint32_t live = A.live[e.x];
            if (live == 0u) continue;
            const int row0 = A.tabs[e.x].varRow0[e.y];
            const uint32_t* c = A.counts + A.rowBase[e.x] + row0;
            const float fl = (float)live;
            uint32_t cmin = 0xffffffffu, cmax = 0u;
            float hl = 0.0f;
            for (int q0 = 0; q0 < nw; q0 += 4) {
                bool pr[4];
                uint32_t cq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = q0 + k;
                    pr[k] = q < nw && ((d[q] >> lane) & 1u);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) cq[k] = pr[k] ? c[(q0 + k) * 32 + lane] : 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!pr[k]) continue;
                    cmin = min(cmin, cq[k]);
                    cmax = max(cmax, cq[k]);
                    if (cq[k]) {
                        const float p = (float)cq[k] / fl;
                        hl -= p * log2f(p);
                    }
                }
            }
            cmin = warp_min(cmin);
            cmax = warp_max(cmax);
            hl = warp_sum_f32(hl);
            bal += (float)s * ((float)cmin / fl);
            top += (float)cmax / fl;
            ent += hl / ls;
            liv += log2f(1.0f + fl) / 32.0f;
            ++cnt;
        }
        if (lane == 0) {
            const float inv = cnt ? 1.0f / (float)cnt : 0.0f;
            f[0] = (float)s / (float)A.varD0[v];
            f[1] = ls / 8.0f;
            f[2] = (float)A.deg[v] / (float)A.degmax;
            f[3] = bal * inv;
            f[4] = top * inv;
            f[5] = ent * inv;
            f[6] = liv * inv;
            f[7] = (float)s / (float)smax;
        }
    }
}

// Offsets of the layers in the flat weight vector.
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kNH * kNF;
constexpr int oW2 = oB1 + kNH;
constexpr int oB2 = oW2 + kNH * kNH;
constexpr int oW3 = oB2 + kNH;
constexpr int oB3 = oW3 + kNH;

// Scores of n rows of X: one warp per row, lane j holding hidden units j and
// j + 32 of both layers; layer-1 outputs reach the other lanes by shuffles.
// Weights sit in shared memory transposed (input-major), so that the lanes of
// a warp read consecutive words.
__global__ void ct_mlp_forward_kernel(const float* __restrict__ w, const float* __restrict__ X, int n,
                                      float* __restrict__ out) {
    __shared__ float w1t[kNF * kNH];  // [i][j] = W1[j][i]
    __shared__ float w2t[kNH * kNH];  // [i][j] = W2[j][i]
    __shared__ float bias1[kNH], bias2[kNH], w3[kNH];
    for (int q = threadIdx.x; q < kNF * kNH; q += blockDim.x) {
        const int j = q / kNF, i = q % kNF;
        w1t[i * kNH + j] = w[oW1 + q];
    }
    for (int q = threadIdx.x; q < kNH * kNH; q += blockDim.x) {
        const int j = q / kNH, i = q % kNH;
        w2t[i * kNH + j] = w[oW2 + q];
    }
    for (int q = threadIdx.x; q < kNH; q += blockDim.x) {
        bias1[q] = w[oB1 + q];
        bias2[q] = w[oB2 + q];
        w3[q] = w[oW3 + q];
    }
    __syncthreads();
    const float b3 = w[oB3];
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int s = gwarp; s < n; s += nwarps) {
        float x[kNF];
#pragma unroll
        for (int i = 0; i < kNF; ++i) x[i] = X[(size_t)s * kNF + i];
        float ha = bias1[lane], hb = bias1[lane + 32];
#pragma unroll
        for (int i = 0; i < kNF; ++i) {
            ha += w1t[i * kNH + lane] * x[i];
            hb += w1t[i * kNH + lane + 32] * x[i];
        }
        ha = fmaxf(ha, 0.0f);
        hb = fmaxf(hb, 0.0f);
        float za = bias2[lane], zb = bias2[lane + 32];
#pragma unroll 8
        for (int i = 0; i < kNH; ++i) {
            const float hi = __shfl_sync(0xffffffffu, i < 32 ? ha : hb, i & 31);
            za += w2t[i * kNH + lane] * hi;
            zb += w2t[i * kNH + lane + 32] * hi;
        }
        float o = w3[lane] * fmaxf(za, 0.0f) + w3[lane + 32] * fmaxf(zb, 0.0f);
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) o += __shfl_xor_sync(0xffffffffu, o, k);
        if (lane == 0) out[s] = o + b3;
    }
}

struct TrainArgs {
    float* w;             // [kNW] in/out
    float* m;             // [kNW] in/out
    float* v;             // [kNW] in/out
    const float* X;       // [n][kNF]
    const float* y;       // [n]
    const int32_t* order; // [epochs][n]
    float* epochLoss;     // [epochs]
    float* grad;          // grad-only mode: [kNW] gradient of the first batch
    int64_t t0;           // Adam steps before this launch
    int32_t n, epochs, batch;
    float lr;
    int32_t gradOnly;
};

constexpr int kTrainThreads = 256;

// Shared-memory layout of the training CTA (floats).
constexpr int sW = 0, sM = sW + kNW, sV = sM + kNW, sX = sV + kNW, sY = sX + kTrainBatch * kNF,
              sH1 = sY + kTrainBatch, sH2 = sH1 + kTrainBatch * kNH, sD1 = sH2 + kTrainBatch * kNH,
              sOut = sD1 + kTrainBatch * kNH, sRed = sOut + kTrainBatch, sTotal = sRed + kTrainThreads;
constexpr size_t kTrainSmem = (size_t)sTotal * sizeof(float);

__device__ __forceinline__ void adam(float* w, float* m, float* v, int i, float g, float lr, float c1, float c2) {
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void __launch_bounds__(kTrainThreads, 1) ct_mlp_train_kernel(const TrainArgs A) {
    extern __shared__ float sm[];
    float* W = sm + sW;
    float* M = sm + sM;
    float* V = sm + sV;
    float* xb = sm + sX;
    float* yb = sm + sY;
    float* H1 = sm + sH1;  // activations of layer 1, then kept for the layer-1 mask
    float* H2 = sm + sH2;  // activations of layer 2, then dL/dz2
    float* D1 = sm + sD1;  // dL/dz1
    float* dout = sm + sOut;
    float* red = sm + sRed;
    const int tid = threadIdx.x;
    for (int i = tid; i < kNW; i += kTrainThreads) {
        W[i] = A.w[i];
        M[i] = A.m[i];
        V[i] = A.v[i];
    }
    __syncthreads();
    int64_t t = A.t0;
    const int epochs = A.gradOnly ? 1 : A.epochs;
    for (int e = 0; e < epochs; ++e) {
        const int32_t* order = A.order + (size_t)e * A.n;
        float lossSum = 0.0f;
        int nb = 0;
        const int nLast = A.gradOnly ? min(A.n, A.batch) : A.n;
        for (int s0 = 0; s0 < nLast; s0 += A.batch) {
            const int b = min(A.batch, nLast - s0);
            for (int i = tid; i < b * kNF; i += kTrainThreads) xb[i] = A.X[(size_t)order[s0 + i / kNF] * kNF + i % kNF];
            for (int i = tid; i < b; i += kTrainThreads) yb[i] = A.y[order[s0 + i]];
            __syncthreads();
            // forward
            for (int q = tid; q < b * kNH; q += kTrainThreads) {
                const int s = q / kNH, j = q % kNH;
                float acc = W[oB1 + j];
                for (int i = 0; i < kNF; ++i) acc += W[oW1 + j * kNF + i] * xb[s * kNF + i];
                H1[q] = fmaxf(acc, 0.0f);
            }
            __syncthreads();
            for (int q = tid; q < b * kNH; q += kTrainThreads) {
                const int s = q / kNH, j = q % kNH;
                float acc = W[oB2 + j];
                for (int i = 0; i < kNH; ++i) acc += W[oW2 + j * kNH + i] * H1[s * kNH + i];
                H2[q] = fmaxf(acc, 0.0f);
            }
            __syncthreads();
            float part = 0.0f;
            for (int s = tid; s < b; s += kTrainThreads) {
                float o = W[oB3];
                for (int j = 0; j < kNH; ++j) o += W[oW3 + j] * H2[s * kNH + j];
                const float r = o - yb[s];
                dout[s] = r / (float)b;
                part += r * r;
            }
            red[tid] = part;
            __syncthreads();
            for (int o = kTrainThreads / 2; o > 0; o >>= 1) {
                if (tid < o) red[tid] += red[tid + o];
                __syncthreads();
            }
            const float loss = red[0] / (2.0f * (float)b);
            ++t;
            const float c1 = 1.0f - powf(0.9f, (float)t);
            const float c2 = 1.0f - powf(0.999f, (float)t);
            // layer 3 gradients (need the layer-2 activations), then dL/dz2 in place
            float g3 = 0.0f;
            if (tid < kNH) {
                for (int s = 0; s < b; ++s) g3 += dout[s] * H2[s * kNH + tid];
            } else if (tid == kNH) {
                for (int s = 0; s < b; ++s) g3 += dout[s];
            }
            __syncthreads();
            for (int q = tid; q < b * kNH; q += kTrainThreads) {
                const int s = q / kNH, j = q % kNH;
                H2[q] = H2[q] > 0.0f ? dout[s] * W[oW3 + j] : 0.0f;
            }
            __syncthreads();
            if (tid <= kNH) {
                const int i = tid < kNH ? oW3 + tid : oB3;
                if (A.gradOnly) A.grad[i] = g3;
                else adam(W, M, V, i, g3, A.lr, c1, c2);
            }
            // dL/dz1 with the old W2
            for (int q = tid; q < b * kNH; q += kTrainThreads) {
                const int s = q / kNH, i = q % kNH;
                float acc = 0.0f;
                if (H1[q] > 0.0f)
                    for (int j = 0; j < kNH; ++j) acc += H2[s * kNH + j] * W[oW2 + j * kNH + i];
                D1[q] = acc;
            }
            __syncthreads();
            // layer 2 gradients and update
            for (int q = tid; q < kNH * kNH + kNH; q += kTrainThreads) {
                float g = 0.0f;
                if (q < kNH * kNH) {
                    const int j = q / kNH, i = q % kNH;
                    for (int s = 0; s < b; ++s) g += H2[s * kNH + j] * H1[s * kNH + i];
                    if (A.gradOnly) A.grad[oW2 + q] = g;
                    else adam(W, M, V, oW2 + q, g, A.lr, c1, c2);
                } else {
                    const int j = q - kNH * kNH;
                    for (int s = 0; s < b; ++s) g += H2[s * kNH + j];
                    if (A.gradOnly) A.grad[oB2 + j] = g;
                    else adam(W, M, V, oB2 + j, g, A.lr, c1, c2);
                }
            }
            // layer 1 gradients and update
            for (int q = tid; q < kNH * kNF + kNH; q += kTrainThreads) {
                float g = 0.0f;
                if (q < kNH * kNF) {
                    const int j = q / kNF, i = q % kNF;
                    for (int s = 0; s < b; ++s) g += D1[s * kNH + j] * xb[s * kNF + i];
                    if (A.gradOnly) A.grad[oW1 + q] = g;
                    else adam(W, M, V, oW1 + q, g, A.lr, c1, c2);
                } else {
                    const int j = q - kNH * kNF;
                    for (int s = 0; s < b; ++s) g += D1[s * kNH + j];
                    if (A.gradOnly) A.grad[oB1 + j] = g;
                    else adam(W, M, V, oB1 + j, g, A.lr, c1, c2);
                }
            }
            __syncthreads();
            lossSum += loss;
            ++nb;
        }
        if (tid == 0) A.epochLoss[e] = nb ? lossSum / (float)nb : 0.0f;
    }
    if (A.gradOnly) return;
    for (int i = tid; i < kNW; i += kTrainThreads) {
        A.w[i] = W[i];
        A.m[i] = M[i];
        A.v[i] = V[i];
    }
}

template <typename T>
int f_alloc(FeatView* f, T** p, size_t n) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("features: cudaMalloc: %s", cudaGetErrorString(e));
        return CT_ERR_OOM;
    }
    f->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return CT_OK;
}

template <typename T>
int f_upload(T* dst, const std::vector<T>& src) {
    if (src.empty()) return CT_OK;
    CT_CUDA(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// feature view
// ---------------------------------------------------------------------------
int ct_feat_view_build(FeatView* f, int nodes, const std::vector<std::vector<int>>& scopes,
                       const std::vector<int>& tableR, const std::vector<int>& tableSeg,
                       const std::vector<int32_t>& varOff, const std::vector<int32_t>& varNW,
                       const std::vector<int32_t>& varD0, int DWg) {
    const int T = (int)scopes.size();
    const int V = (int)varOff.size();
    const int nt = nodes * T, nv = nodes * V;
    f->nodes = nodes;
    f->T = T;
    f->V = V;
    f->nt = nt;
    f->nv = nv;
    std::vector<int32_t> rowBase(nt + 1, 0), unitBase(nt + 1, 0), scopeBase(nt + 1, 0), scopeOff, vOff(nv), vNW(nv),
        vD0(nv), deg(nv, 0), adjBase(nv + 1, 0);
    std::vector<int2> adj;
    std::vector<std::vector<int2>> perVar(V);
    for (int k = 0; k < T; ++k)
        for (int i = 0; i < (int)scopes[k].size(); ++i) perVar[scopes[k][i]].push_back(make_int2(k, i));
    int degmax = 1;
    for (int v = 0; v < V; ++v) degmax = std::max(degmax, (int)perVar[v].size());
    for (int n = 0; n < nodes; ++n) {
        for (int k = 0; k < T; ++k) {
            const int t = n * T + k;
            rowBase[t + 1] = rowBase[t] + tableR[k];
            int sw = 0;
            for (int v : scopes[k]) sw += varNW[v];
            unitBase[t + 1] = unitBase[t] + tableSeg[k] * sw;
            scopeBase[t + 1] = scopeBase[t] + (int)scopes[k].size();
            for (int v : scopes[k]) scopeOff.push_back(varOff[v] + n * DWg);
        }
        for (int v = 0; v < V; ++v) {
            const int g = n * V + v;
            vOff[g] = varOff[v] + n * DWg;
            vNW[g] = varNW[v];
            vD0[g] = varD0[v];
            deg[g] = (int)perVar[v].size();
            for (const int2& e : perVar[v]) adj.push_back(make_int2(n * T + e.x, e.y));
            adjBase[g + 1] = (int)adj.size();
        }
    }
    f->degmax = degmax;
    f->totalUnits = unitBase[nt];
    f->totalRows = rowBase[nt];
    int st;
    if ((st = f_alloc(f, &f->rowBase, nt + 1)) != CT_OK || (st = f_alloc(f, &f->unitBase, nt + 1)) != CT_OK ||
        (st = f_alloc(f, &f->scopeBase, nt + 1)) != CT_OK || (st = f_alloc(f, &f->scopeOff, scopeOff.size())) != CT_OK ||
        (st = f_alloc(f, &f->adjBase, nv + 1)) != CT_OK || (st = f_alloc(f, &f->adj, adj.size())) != CT_OK ||
        (st = f_alloc(f, &f->varOff, nv)) != CT_OK || (st = f_alloc(f, &f->varNW, nv)) != CT_OK ||
        (st = f_alloc(f, &f->varD0, nv)) != CT_OK || (st = f_alloc(f, &f->deg, nv)) != CT_OK ||
        (st = f_alloc(f, &f->counts, rowBase[nt])) != CT_OK || (st = f_alloc(f, &f->live, nt)) != CT_OK ||
        (st = f_alloc(f, &f->feat, (size_t)nv * kNF)) != CT_OK || (st = f_alloc(f, &f->scores, nv)) != CT_OK)
        return st;
    if ((st = f_upload(f->rowBase, rowBase)) != CT_OK || (st = f_upload(f->unitBase, unitBase)) != CT_OK ||
        (st = f_upload(f->scopeBase, scopeBase)) != CT_OK || (st = f_upload(f->scopeOff, scopeOff)) != CT_OK ||
        (st = f_upload(f->adjBase, adjBase)) != CT_OK || (st = f_upload(f->adj, adj)) != CT_OK ||
        (st = f_upload(f->varOff, vOff)) != CT_OK || (st = f_upload(f->varNW, vNW)) != CT_OK ||
        (st = f_upload(f->varD0, vD0)) != CT_OK || (st = f_upload(f->deg, deg)) != CT_OK)
        return st;
    if (cudaHostAlloc((void**)&f->h_scores, std::max(nv, 1) * sizeof(float), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        ct_set_error("features: pinned scores");
        return CT_ERR_OOM;
    }
    return CT_OK;
}

void ct_feat_view_free(FeatView* f) {
    if (!f) return;
    for (void* p : f->allocs) cudaFree(p);
    f->allocs.clear();
    if (f->h_scores) cudaFreeHost(f->h_scores);
    f->h_scores = nullptr;
    cudaGetLastError();
}

int ct_feat_compute(FeatView* f, const TableDev* d_tabs, const uint32_t* dom, const uint8_t* nodeActive,
                    cudaStream_t s) {
    if (!f->counts) {
        ct_set_error("features: view not built");
        return CT_ERR_STATE;
    }
    FeatArgs A;
    A.tabs = d_tabs;
    A.dom = dom;
    A.nodeActive = nodeActive;
    A.rowBase = f->rowBase;
    A.unitBase = f->unitBase;
    A.scopeBase = f->scopeBase;
    A.scopeOff = f->scopeOff;
    A.adjBase = f->adjBase;
    A.adj = f->adj;
    A.varOff = f->varOff;
    A.varNW = f->varNW;
    A.varD0 = f->varD0;
    A.deg = f->deg;
    A.counts = f->counts;
    A.live = f->live;
    A.feat = f->feat;
    A.nt = f->nt;
    A.nv = f->nv;
    A.T = f->T;
    A.V = f->V;
    A.degmax = f->degmax;
    A.totalUnits = f->totalUnits;
    CT_CUDA(cudaMemsetAsync(f->counts, 0, sizeof(uint32_t) * (size_t)std::max(f->totalRows, 1), s));
    CT_CUDA(cudaMemsetAsync(f->live, 0, sizeof(uint32_t) * (size_t)std::max(f->nt, 1), s));
    int sms = 0, dev = 0;
    CT_CUDA(cudaGetDevice(&dev));
    CT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int warps = std::max(1, f->totalUnits);
    const int grid = std::max(1, std::min((warps + 7) / 8, sms * 8));
    if (f->totalUnits > 0) {
        ct_counts_kernel<<<grid, 256, 0, s>>>(A);
        CT_CUDA(cudaGetLastError());
    }
    const int perNode = (f->V + 7) / 8;
    ct_features_kernel<<<f->nodes * std::max(perNode, 1), 256, 0, s>>>(A, std::max(perNode, 1));
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int ct_feat_scores(FeatView* f, const ct_mlp* mlp, cudaStream_t s) {
    const int n = f->nv;
    const int grid = std::max(1, std::min((n + 7) / 8, 1024));
    ct_mlp_forward_kernel<<<grid, 256, 0, s>>>(mlp->d_w, f->feat, n, f->scores);
    CT_CUDA(cudaGetLastError());
    CT_CUDA(cudaMemcpyAsync(f->h_scores, f->scores, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    return CT_OK;
}

// ---------------------------------------------------------------------------
// C ABI: the scoring network
// ---------------------------------------------------------------------------
namespace {

int mlp_reset(ct_mlp* m, const float* w_host) {
    CT_CUDA(cudaMemcpyAsync(m->d_w, w_host, kNW * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    CT_CUDA(cudaMemsetAsync(m->d_m, 0, kNW * sizeof(float), m->stream));
    CT_CUDA(cudaMemsetAsync(m->d_v, 0, kNW * sizeof(float), m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    m->t = 0;
    return CT_OK;
}

// Device copies of a host array (freed by the caller with cudaFree).
template <typename T>
int to_device(const T* h, size_t n, T** d, cudaStream_t s) {
    *d = nullptr;
    cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(*d, h, n * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        if (*d) cudaFree(*d);
        *d = nullptr;
        return ct_cuda_fail(e, "training data upload");
    }
    return CT_OK;
}

int run_train(ct_mlp* m, const float* x_host, const float* y_host, int64_t n, const int32_t* orders, int epochs,
              int batch, float lr, bool gradOnly, float* loss_out, float* grad_host) {
    float *dX = nullptr, *dY = nullptr, *dLoss = nullptr, *dGrad = nullptr;
    int32_t* dOrd = nullptr;
    std::vector<int32_t> ident;
    if (gradOnly) {
        ident.resize((size_t)n);
        for (int64_t i = 0; i < n; ++i) ident[(size_t)i] = (int32_t)i;
        orders = ident.data();
    }
    int st = to_device(x_host, (size_t)n * kNF, &dX, m->stream);
    if (st == CT_OK) st = to_device(y_host, (size_t)n, &dY, m->stream);
    if (st == CT_OK) st = to_device(orders, (size_t)n * (gradOnly ? 1 : epochs), &dOrd, m->stream);
    cudaError_t e = cudaSuccess;
    if (st == CT_OK) {
        e = cudaMalloc((void**)&dLoss, sizeof(float) * (size_t)std::max(epochs, 1));
        if (e == cudaSuccess) e = cudaMalloc((void**)&dGrad, sizeof(float) * kNW);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ct_mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
        if (e == cudaSuccess) {
            TrainArgs A;
            A.w = m->d_w;
            A.m = m->d_m;
            A.v = m->d_v;
            A.X = dX;
            A.y = dY;
            A.order = dOrd;
            A.epochLoss = dLoss;
            A.grad = dGrad;
            A.t0 = m->t;
            A.n = (int32_t)n;
            A.epochs = gradOnly ? 1 : epochs;
            A.batch = batch;
            A.lr = lr;
            A.gradOnly = gradOnly ? 1 : 0;
            ct_mlp_train_kernel<<<1, kTrainThreads, kTrainSmem, m->stream>>>(A);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && loss_out)
            e = cudaMemcpyAsync(loss_out, dLoss, sizeof(float) * (size_t)(gradOnly ? 1 : epochs), cudaMemcpyDeviceToHost,
                                m->stream);
        if (e == cudaSuccess && gradOnly && grad_host)
            e = cudaMemcpyAsync(grad_host, dGrad, sizeof(float) * kNW, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = ct_cuda_fail(e, "ct_mlp training kernel");
    }
    if (dX) cudaFree(dX);
    if (dY) cudaFree(dY);
    if (dOrd) cudaFree(dOrd);
    if (dLoss) cudaFree(dLoss);
    if (dGrad) cudaFree(dGrad);
    if (st == CT_OK && !gradOnly) {
        const int64_t per = (n + batch - 1) / batch;
        m->t += per * epochs;
    }
    return st;
}

}  // namespace

extern "C" int ct_mlp_create(const float* weights_host, void* cuda_stream, ct_mlp** out) {
    if (!out || !weights_host) {
        ct_set_error("ct_mlp_create: null argument");
        return CT_ERR_ARG;
    }
    *out = nullptr;
    ct_mlp* m = new (std::nothrow) ct_mlp();
    if (!m) return CT_ERR_OOM;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        m->ownStream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->d_w, kNW * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->d_m, kNW * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->d_v, kNW * sizeof(float));
    int st = e == cudaSuccess ? mlp_reset(m, weights_host) : ct_cuda_fail(e, "ct_mlp_create");
    if (st != CT_OK) {
        ct_mlp_destroy(m);
        return st;
    }
    *out = m;
    return CT_OK;
}

extern "C" int ct_mlp_set_weights(ct_mlp* m, const float* weights_host) {
    if (!m || !weights_host) {
        ct_set_error("ct_mlp_set_weights: null argument");
        return CT_ERR_ARG;
    }
    return mlp_reset(m, weights_host);
}

extern "C" int ct_mlp_get_weights(ct_mlp* m, float* weights_host) {
    if (!m || !weights_host) {
        ct_set_error("ct_mlp_get_weights: null argument");
        return CT_ERR_ARG;
    }
    CT_CUDA(cudaMemcpyAsync(weights_host, m->d_w, kNW * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    CT_CUDA(cudaStreamSynchronize(m->stream));
    return CT_OK;
}

extern "C" int ct_mlp_forward(ct_mlp* m, const float* x_dev, int64_t n, float* scores_dev) {
    if (!m || (n > 0 && (!x_dev || !scores_dev)) || n < 0 || n > 0x7fffffffLL) {
        ct_set_error("ct_mlp_forward: bad argument");
        return CT_ERR_ARG;
    }
    if (n == 0) return CT_OK;
    const int grid = (int)std::min<int64_t>((n + 7) / 8, 4096);
    ct_mlp_forward_kernel<<<grid, 256, 0, m->stream>>>(m->d_w, x_dev, (int)n, scores_dev);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

extern "C" int ct_mlp_grad(ct_mlp* m, const float* x_host, const float* y_host, int n, float* loss_out,
                           float* grad_host) {
    if (!m || !x_host || !y_host || !grad_host || n < 1 || n > kTrainBatch) {
        ct_set_error("ct_mlp_grad: bad argument (1 <= n <= %d)", kTrainBatch);
        return CT_ERR_ARG;
    }
    return run_train(m, x_host, y_host, n, nullptr, 1, n, 0.0f, true, loss_out, grad_host);
}

extern "C" int ct_mlp_train(ct_mlp* m, const float* x_host, const float* y_host, int64_t n, const int32_t* orders_host,
                            int epochs, int batch, float lr, float* epoch_loss_host) {
    if (!m || !x_host || !y_host || !orders_host || n < 1 || n > 0x7fffffffLL || epochs < 1 || batch < 1 ||
        batch > kTrainBatch || !(lr > 0.0f)) {
        ct_set_error("ct_mlp_train: bad argument (1 <= batch <= %d, epochs >= 1, lr > 0)", kTrainBatch);
        return CT_ERR_ARG;
    }
    for (int64_t i = 0; i < n * epochs; ++i) {
        if (orders_host[i] < 0 || orders_host[i] >= n) {
            ct_set_error("ct_mlp_train: order entry %lld out of range", (long long)i);
            return CT_ERR_ARG;
        }
    }
    return run_train(m, x_host, y_host, n, orders_host, epochs, batch, lr, false, epoch_loss_host, nullptr);
}

extern "C" int ct_mlp_destroy(ct_mlp* m) {
    if (!m) return CT_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->d_w) cudaFree(m->d_w);
    if (m->d_m) cudaFree(m->d_m);
    if (m->d_v) cudaFree(m->d_v);
    if (m->ownStream && m->stream) cudaStreamDestroy(m->stream);
    cudaGetLastError();
    delete m;
    return CT_OK;
}
