// mn_learned.cuh -- learned choice of the matching order per seed.
//
// A small regression network predicts the enumeration work of a seed under
// each candidate matching order (NCAND plans per (query, seed edge), the
// paper's order first); the order with the smallest prediction is used.  The
// choice never changes what is enumerated -- every candidate order is a
// connected order of the same query -- only how much work it takes.
//
// Network: 16 features -> 128 -> 128 -> 1, ReLU, weights and activations in
// BF16 with FP32 accumulation (inference: mma.sync m16n8k16 on the tensor
// cores), FP32 master weights, mean squared error on log2(1 + work), Adam
// (Kingma & Ba, 2015).  Training data are logged by the enumerator itself:
// per seed the SM cycles spent on it (summed over the seed's own unit and
// every subtree split off from it).
#pragma once
#include <cuda_bf16.h>
#include "mn_device.cuh"

namespace mn {

constexpr int NF = 16, NH = 128;
// FP32 parameter block: W1[NF][NH], b1[NH], W2[NH][NH], b2[NH], w3[NH], b3
constexpr int P_W1 = 0, P_B1 = P_W1 + NF * NH, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH,
              P_W3 = P_B2 + NH, P_B3 = P_W3 + NH, P_COUNT = P_B3 + 1;

// ------------------------------------------------------------------ features

struct FeatParams {
    const unsigned long long *seeds;
    const uint32_t *nseeds;
    uint32_t seed_cap;
    uint32_t all_candidates;            // 1: NCAND rows per seed; 0: the seed's own candidate
    const uint32_t *ring_src, *ring_dst;
    const uint8_t *r_label;
    const uint32_t *offs[2];
    uint32_t L, cap_mask;
    uint32_t *const *debi;
    const Plan *plans;
    const uint32_t *temporal;           // per query: 1 if it has precedence pairs
    __nv_bfloat16 *X;                   // rows of NF features
};

__device__ __forceinline__ float lg(uint32_t x) { return log2f(1.0f + (float)x); }

// Features of (seed, candidate order): the seed's label-slice degrees, total
// degrees, DEBI popcount, query shape and the branching of the order's first
// two steps.
__global__ void k_features(FeatParams p)
{
    const uint32_t n = min(*p.nseeds, p.seed_cap);
    const uint32_t per = p.all_candidates ? NCAND : 1;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n * per; r += gridDim.x * blockDim.x) {
        const uint32_t s = r / per;
        const unsigned long long sd = p.seeds[s];
        const uint32_t s32 = (uint32_t)(sd >> 32), q = (uint32_t)(sd >> 8) & 0xffffu;
        const uint32_t j = (uint32_t)sd & 0xffu;
        const uint32_t k = p.all_candidates ? r % NCAND : (uint32_t)(sd >> 24) & (NCAND - 1);
        const uint32_t slot = s32 & p.cap_mask;
        const uint32_t vs = p.ring_src[slot], vd = p.ring_dst[slot], lab = p.r_label[slot];
        const uint32_t L = p.L;
        const uint32_t *o0 = p.offs[0], *o1 = p.offs[1];
        auto seg = [&](const uint32_t *o, uint32_t v, uint32_t l) { return o[v * L + l + 1] - o[v * L + l]; };
        auto all = [&](const uint32_t *o, uint32_t v) { return o[v * L + L] - o[v * L]; };
        const Plan &P = p.plans[(q * MN_MAX_QE + j) * NCAND + k];
        float f[NF];
        f[0] = lg(seg(o0, vs, lab));
        f[1] = lg(seg(o1, vs, lab));
        f[2] = lg(seg(o0, vd, lab));
        f[3] = lg(seg(o1, vd, lab));
        f[4] = lg(all(o0, vs));
        f[5] = lg(all(o1, vd));
        f[6] = (float)__popc(p.debi[q][slot]) / 16.0f;
        f[7] = (float)j / (float)P.ne;
        f[8] = (float)P.nv / 16.0f;
        f[9] = (float)P.ne / 16.0f;
        f[10] = (float)(P.ne + 1 - P.nv) / (float)P.ne;
        f[11] = (float)p.temporal[q];
        // branching of steps 1 and 2 when they extend from a seed endpoint
        float br[2] = {0.f, 0.f};
        for (int st = 1; st <= 2 && st < P.nsteps; st++) {
            const Step &S = P.step[st];
            if (S.kind != K_EXTEND || (S.from != P.seed_src && S.from != P.seed_dst)) continue;
            const uint32_t v = S.from == P.seed_src ? vs : vd;
            const uint32_t *o = S.dir ? o1 : o0;
            br[st - 1] = lg(S.label >= 0 ? seg(o, v, (uint32_t)S.label) : all(o, v));
        }
        f[12] = br[0];
        f[13] = br[1];
        f[14] = (float)(k & 1);
        f[15] = (float)(k >> 1);
        __nv_bfloat16 *x = p.X + (size_t)r * NF;
        for (int i = 0; i < NF; i++) x[i] = __float2bfloat16_rn(f[i]);
    }
}

// ------------------------------------------------------------------ inference

__device__ __forceinline__ void mma_bf16(float &d0, float &d1, float &d2, float &d3, uint32_t a0,
                                         uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// BF16 copies of the weights, transposed (output-major) for the B operand.
__global__ void k_mlp_pack(const float *P, __nv_bfloat16 *w1t, __nv_bfloat16 *w2t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NF * NH) {                       // w1t[h][f] = W1[f][h]
        const int h = i / NF, f = i % NF;
        w1t[i] = __float2bfloat16_rn(P[P_W1 + f * NH + h]);
    }
    if (i < NH * NH) {                       // w2t[o][h] = W2[h][o]
        const int o = i / NH, h = i % NH;
        w2t[i] = __float2bfloat16_rn(P[P_W2 + h * NH + o]);
    }
}

constexpr int MLP_WARPS = 4;   // 16 rows per warp

// y[r] = w3 . relu(W2^T bf16(relu(W1^T x_r + b1)) + b2) + b3 for rows r < n
// (n read from *n_dev times `per`, or n_host when n_dev is NULL).
__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_forward(
    const __nv_bfloat16 *__restrict__ X, const uint32_t *n_dev, uint32_t per, uint32_t n_host,
    const __nv_bfloat16 *__restrict__ w1t, const __nv_bfloat16 *__restrict__ w2t,
    const float *__restrict__ P, float *__restrict__ y)
{
    __shared__ __align__(16) __nv_bfloat16 sw1[NH * NF];
    __shared__ __align__(16) __nv_bfloat16 sw2[NH * NH];
    __shared__ float sb1[NH], sb2[NH], sw3[NH];
    for (int i = threadIdx.x; i < NH * NF; i += blockDim.x) sw1[i] = w1t[i];
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) sw2[i] = w2t[i];
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        sb1[i] = P[P_B1 + i]; sb2[i] = P[P_B2 + i]; sw3[i] = P[P_W3 + i];
    }
    __syncthreads();
    const uint32_t n = n_dev ? *n_dev * per : n_host;
    const float b3 = P[P_B3];
    const int lane = threadIdx.x & 31, gq = lane >> 2, t4 = lane & 3;
    const uint32_t *x32 = reinterpret_cast<const uint32_t *>(X);
    const uint32_t *s1 = reinterpret_cast<const uint32_t *>(sw1);
    const uint32_t *s2 = reinterpret_cast<const uint32_t *>(sw2);
    for (uint32_t rb = (blockIdx.x * MLP_WARPS + (threadIdx.x >> 5)) * 16; rb < n;
         rb += gridDim.x * MLP_WARPS * 16) {
        const uint32_t r0 = rb + gq, r1 = rb + gq + 8;
        // A fragment of X (16 rows x 16 features)
        const uint32_t a0 = r0 < n ? x32[r0 * (NF / 2) + t4] : 0u;
        const uint32_t a1 = r1 < n ? x32[r1 * (NF / 2) + t4] : 0u;
        const uint32_t a2 = r0 < n ? x32[r0 * (NF / 2) + t4 + 4] : 0u;
        const uint32_t a3 = r1 < n ? x32[r1 * (NF / 2) + t4 + 4] : 0u;
        // layer 1 -> A fragments of layer 2 (k-block m = n-tiles 2m, 2m+1)
        uint32_t h[NH / 16][4];
#pragma unroll
        for (int nt = 0; nt < NH / 8; nt++) {
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            const int col = nt * 8 + gq;
            mma_bf16(c0, c1, c2, c3, a0, a1, a2, a3, s1[col * (NF / 2) + t4], s1[col * (NF / 2) + t4 + 4]);
            const int oc = nt * 8 + 2 * t4;
            c0 = fmaxf(c0 + sb1[oc], 0.f); c1 = fmaxf(c1 + sb1[oc + 1], 0.f);
            c2 = fmaxf(c2 + sb1[oc], 0.f); c3 = fmaxf(c3 + sb1[oc + 1], 0.f);
            const int m = nt >> 1, half = nt & 1;
            h[m][half * 2 + 0] = pack_bf16(c0, c1);
            h[m][half * 2 + 1] = pack_bf16(c2, c3);
        }
        // layer 2 and the output dot product
        float y0 = 0.f, y1 = 0.f;
#pragma unroll 4
        for (int nt = 0; nt < NH / 8; nt++) {
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            const int col = nt * 8 + gq;
#pragma unroll
            for (int m = 0; m < NH / 16; m++)
                mma_bf16(c0, c1, c2, c3, h[m][0], h[m][1], h[m][2], h[m][3],
                         s2[col * (NH / 2) + m * 8 + t4], s2[col * (NH / 2) + m * 8 + t4 + 4]);
            const int oc = nt * 8 + 2 * t4;
            c0 = fmaxf(c0 + sb2[oc], 0.f); c1 = fmaxf(c1 + sb2[oc + 1], 0.f);
            c2 = fmaxf(c2 + sb2[oc], 0.f); c3 = fmaxf(c3 + sb2[oc + 1], 0.f);
            y0 += c0 * sw3[oc] + c1 * sw3[oc + 1];
            y1 += c2 * sw3[oc] + c3 * sw3[oc + 1];
        }
        y0 += __shfl_xor_sync(FULL, y0, 1); y0 += __shfl_xor_sync(FULL, y0, 2);
        y1 += __shfl_xor_sync(FULL, y1, 1); y1 += __shfl_xor_sync(FULL, y1, 2);
        if (t4 == 0) {
            if (r0 < n) y[r0] = y0 + b3;
            if (r1 < n) y[r1] = y1 + b3;
        }
    }
}

// ------------------------------------------------------------------ training

constexpr int TR_ROWS = 16, TR_THREADS = NH;
constexpr size_t TR_SMEM = sizeof(float) * ((size_t)P_COUNT + TR_ROWS * (NF + 4 * NH + 2));

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Gradient of the mean squared error over rows [0, n) with the same BF16
// rounding as inference (weights and the layer-1 activations), accumulated
// per block in shared memory and added to g[] (FP32); the loss sum goes to
// *loss.  Thread h owns hidden unit h.
__global__ void __launch_bounds__(TR_THREADS) k_mlp_grad(
    const __nv_bfloat16 *__restrict__ X, const float *__restrict__ T, uint32_t n,
    const float *__restrict__ P, float *__restrict__ G, float *__restrict__ loss)
{
    extern __shared__ float sm[];
    float *dG = sm;                                  // P_COUNT
    float *x = dG + P_COUNT;                         // [TR_ROWS][NF]
    float *h1 = x + TR_ROWS * NF;                    // [TR_ROWS][NH] bf16-rounded relu
    float *h2 = h1 + TR_ROWS * NH;                   // [TR_ROWS][NH] relu
    float *d2 = h2 + TR_ROWS * NH;                   // dZ2
    float *d1 = d2 + TR_ROWS * NH;                   // dZ1
    float *dy = d1 + TR_ROWS * NH;                   // [TR_ROWS]
    float *yy = dy + TR_ROWS;                        // [TR_ROWS]
    const int h = threadIdx.x;
    for (int i = h; i < P_COUNT; i += blockDim.x) dG[i] = 0.f;
    float lsum = 0.f;
    const float inv_n = 1.0f / (float)max(n, 1u);
    __syncthreads();
    for (uint32_t r0 = blockIdx.x * TR_ROWS; r0 < n; r0 += gridDim.x * TR_ROWS) {
        const int rows = (int)min((uint32_t)TR_ROWS, n - r0);
        for (int i = h; i < TR_ROWS * NF; i += blockDim.x)
            x[i] = i / NF < rows ? __bfloat162float(X[(size_t)(r0 + i / NF) * NF + i % NF]) : 0.f;
        __syncthreads();
        for (int r = 0; r < rows; r++) {             // layer 1 (unit h)
            float z = P[P_B1 + h];
            for (int f = 0; f < NF; f++) z += x[r * NF + f] * bf16r(P[P_W1 + f * NH + h]);
            h1[r * NH + h] = z > 0.f ? bf16r(z) : 0.f;
        }
        __syncthreads();
        for (int r = 0; r < rows; r++) {             // layer 2 (unit h)
            float z = P[P_B2 + h];
            for (int k = 0; k < NH; k++) z += h1[r * NH + k] * bf16r(P[P_W2 + k * NH + h]);
            h2[r * NH + h] = z > 0.f ? z : 0.f;
        }
        __syncthreads();
        if (h < TR_ROWS) {                           // output and dL/dy
            float v = P[P_B3];
            if (h < rows) {
                for (int k = 0; k < NH; k++) v += h2[h * NH + k] * P[P_W3 + k];
                const float e = v - T[r0 + h];
                dy[h] = 2.f * e * inv_n;
                lsum += e * e;
            } else {
                dy[h] = 0.f;
            }
            yy[h] = v;
        }
        __syncthreads();
        {
            const float w3 = P[P_W3 + h];
            float gw3 = 0.f, gb2 = 0.f;
            for (int r = 0; r < rows; r++) {
                gw3 += dy[r] * h2[r * NH + h];
                const float dz = h2[r * NH + h] > 0.f ? dy[r] * w3 : 0.f;
                d2[r * NH + h] = dz;
                gb2 += dz;
            }
            dG[P_W3 + h] += gw3;
            dG[P_B2 + h] += gb2;
            if (h == 0) for (int r = 0; r < rows; r++) dG[P_B3] += dy[r];
        }
        __syncthreads();
        for (int k = 0; k < NH; k++) {               // dW2[k][h]
            float s = 0.f;
            for (int r = 0; r < rows; r++) s += h1[r * NH + k] * d2[r * NH + h];
            dG[P_W2 + k * NH + h] += s;
        }
        for (int r = 0; r < rows; r++) {             // dZ1[r][h] through W2 row h
            float s = 0.f;
            for (int o = 0; o < NH; o++) s += bf16r(P[P_W2 + h * NH + o]) * d2[r * NH + o];
            d1[r * NH + h] = h1[r * NH + h] > 0.f ? s : 0.f;
        }
        __syncthreads();
        {
            float gb1 = 0.f;
            for (int r = 0; r < rows; r++) gb1 += d1[r * NH + h];
            dG[P_B1 + h] += gb1;
            for (int f = 0; f < NF; f++) {
                float s = 0.f;
                for (int r = 0; r < rows; r++) s += x[r * NF + f] * d1[r * NH + h];
                dG[P_W1 + f * NH + h] += s;
            }
        }
        __syncthreads();
    }
    for (int i = h; i < P_COUNT; i += blockDim.x) atomicAdd(&G[i], dG[i]);
    if (h < TR_ROWS) atomicAdd(loss, lsum * inv_n);
}

// One Adam step (Kingma & Ba 2015) on the FP32 master parameters.
__global__ void k_adam(float *P, const float *G, float *M1, float *M2, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M1[i] + (1.f - b1) * g;
    const float v = b2 * M2[i] + (1.f - b2) * g * g;
    M1[i] = m;
    M2[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// ------------------------------------------------------------------ order choice

// Per seed: the candidate order with the smallest predicted cost, but the
// paper's order (candidate 0) unless the best prediction beats it by at least
// `margin` (log2 units): the paper's order is the fallback.  A seed whose
// predicted cost under the chosen order is at least `split_log2` is flagged
// for pre-splitting (SEED_PRESPLIT; split_log2 = +inf: never).
__global__ void k_pick(unsigned long long *seeds, const uint32_t *nseeds, uint32_t seed_cap,
                       const float *y, float margin, float split_log2)
{
    const uint32_t n = min(*nseeds, seed_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t best = 0;
        const float y0 = y[(size_t)s * NCAND];
        float bv = y0;
        for (uint32_t k = 1; k < NCAND; k++) {
            const float v = y[(size_t)s * NCAND + k];
            if (v < bv) { bv = v; best = k; }
        }
        if (bv > y0 - margin) { best = 0; bv = y0; }
        unsigned long long w = (seeds[s] & ~(0xffull << 24)) | ((unsigned long long)best << 24);
        if (bv >= split_log2) w |= SEED_PRESPLIT;
        seeds[s] = w;
    }
}

// Exploration: a pseudo-random candidate per seed (splitmix64 of seed index
// and round), so that logged work covers every candidate order.
__global__ void k_explore(unsigned long long *seeds, const uint32_t *nseeds, uint32_t seed_cap,
                          unsigned long long round)
{
    const uint32_t n = min(*nseeds, seed_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        unsigned long long z = (round << 32) + s + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const unsigned long long k = z % NCAND;
        seeds[s] = (seeds[s] & ~(0xffull << 24)) | (k << 24);
    }
}

// Append (features of the seed's own order, log2(1 + logged cycles)) to the
// training ring at position *pos (advanced afterwards by k_advance).
__global__ void k_log_samples(const __nv_bfloat16 *X, const unsigned long long *work,
                              const uint32_t *nseeds, uint32_t seed_cap, __nv_bfloat16 *SX,
                              float *ST, const unsigned long long *pos, uint32_t ring)
{
    const uint32_t n = min(*nseeds, seed_cap);
    const unsigned long long base = *pos;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t dst = (uint32_t)((base + s) % ring);
        for (int f = 0; f < NF; f++) SX[(size_t)dst * NF + f] = X[(size_t)s * NF + f];
        ST[dst] = log2f(1.0f + (float)work[s]);
    }
}

__global__ void k_advance(unsigned long long *pos, const uint32_t *nseeds, uint32_t seed_cap)
{
    *pos += min(*nseeds, seed_cap);
}

}  // namespace mn
