// mn_learned.cuh -- learned choice of the matching order per seed.
//
// A small regression network predicts the enumeration work of a seed under
// each candidate matching order (NCAND plans per (query, seed edge), the
// paper's order first); the order with the smallest prediction is used.  The
// choice never changes what is enumerated -- every candidate order is a
// connected order of the same query -- only how much work it takes.
//
// Network: 16 features -> 128 -> 128 -> 1, ReLU, weights and activations in
// BF16 with FP32 accumulation, FP32 master weights, mean squared error on
// log2(1 + work), Adam (Kingma & Ba, 2015).  Inference (k_mlp_forward_tc)
// and the gradient (k_mlp_grad_tc) run on the 5th-generation tensor cores:
// tcgen05.mma from shared-memory operand tiles into TMEM accumulators.
// Training data are logged by the enumerator itself: per seed the SM cycles
// spent on it (summed over the seed's own unit and every subtree split off
// from it).
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

// ------------------------------------------------------------------ inference on tcgen05

// 5th-generation tensor cores: the operands sit in shared memory as K-major
// tiles of 8-row x 16-byte core matrices (no swizzling), the FP32
// accumulators in tensor memory (TMEM, one lane per row), one thread issues
// the MMAs and a commit to an mbarrier tells every thread when they are done.

// Shared-memory matrix descriptor of a K-major operand without swizzling:
// start address, `lbo` bytes between core matrices adjacent along K, `sbo`
// bytes between adjacent 8-row groups; bits 46-48 hold the descriptor
// version (0b001), base offset, address mode and swizzle fields are 0.
__device__ __forceinline__ unsigned long long umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at
// bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(uint32_t m, uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)    // one whole warp
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(dst)), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_relinquish()                            // one whole warp
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) // one whole warp
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B^T (+ D when accumulate), A: M x K, B: N x K, K = 16
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, unsigned long long a_desc,
                                          unsigned long long b_desc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// arrive on *bar once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32w .. 32w + 31), waited for within the same statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major core-matrix tile whose rows
// hold K elements of 2 bytes: core matrices along K are 128 bytes apart
// (LBO), 8-row groups K / 8 * 128 bytes apart (SBO).
__host__ __device__ constexpr uint32_t cm_off(uint32_t row, uint32_t k, uint32_t K)
{
    return (row >> 3) * (K / 8) * 128u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

constexpr uint32_t TC_M = 128;                         // rows per tile = TMEM lanes
constexpr uint32_t TC_B1 = 0;                          // W1^T as B: N = 128 x K = 16
constexpr uint32_t TC_B2 = TC_B1 + NH * NF * 2;        // W2^T as B: N = 128 x K = 128
constexpr uint32_t TC_A1 = TC_B2 + NH * NH * 2;        // X tile: M = 128 x K = 16
constexpr uint32_t TC_A2 = TC_A1 + TC_M * NF * 2;      // bf16(relu(layer 1)): M = 128 x K = 128
constexpr uint32_t TC_VEC = TC_A2 + TC_M * NH * 2;     // b1, b2, w3 (FP32)
constexpr uint32_t TC_SUM = TC_VEC + 3 * NH * 4;       // the second column half's output sums
constexpr uint32_t TC_BAR = TC_SUM + TC_M * 4;         // mbarrier, TMEM base address
constexpr uint32_t TC_SMEM = TC_BAR + 16;
constexpr uint32_t TC_TMEM_COLS = 2 * NH;              // layer 1 in columns [0, 128), layer 2 in [128, 256)
constexpr uint32_t TC_WAIT_POLLS = 1u << 24;

constexpr uint32_t TC_FWD_THREADS = 2 * TC_M;     // two warpgroups: column halves of each row

// y[r] = w3 . relu(W2^T bf16(relu(W1^T x_r + b1)) + b2) + b3 for rows r < n
// (n read from *n_dev times `per`, or n_host when n_dev is NULL); 128 rows
// per tile, tiles strided over the grid (launched with two blocks per SM:
// each holds 256 of the SM's 512 TMEM columns, so one block's epilogue runs
// while the other's MMAs do).  Two warpgroups share the epilogues: warp w
// reads TMEM lanes 32 (w mod 4) .. + 31 (its rows), warpgroup 0 the columns
// 0-63 of each accumulator and warpgroup 1 the columns 64-127; the output
// dot product adds the two halves through shared memory.  *status gets
// ST_TIMEOUT if an MMA completion was not seen within the wait bound (every
// thread still runs every tile, so the block's barriers stay matched).
__global__ void __launch_bounds__(TC_FWD_THREADS, 2) k_mlp_forward_tc(
    const __nv_bfloat16 *__restrict__ X, const uint32_t *n_dev, uint32_t per, uint32_t n_host,
    const __nv_bfloat16 *__restrict__ w1t, const __nv_bfloat16 *__restrict__ w2t,
    const float *__restrict__ P, float *__restrict__ y, uint32_t *status)
{
    extern __shared__ __align__(1024) uint8_t tcs[];
    float *vb1 = reinterpret_cast<float *>(tcs + TC_VEC), *vb2 = vb1 + NH, *vw3 = vb2 + NH;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(tcs + TC_BAR);
    uint32_t *tbase = reinterpret_cast<uint32_t *>(tcs + TC_BAR + 8);
    float *half_sum = reinterpret_cast<float *>(tcs + TC_SUM);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const uint32_t row = tid & (TC_M - 1), wg = tid / TC_M;   // this thread's tile row and column half
    const uint32_t n = n_dev ? *n_dev * per : n_host;
    if (blockIdx.x * TC_M >= n) return;                // the whole block leaves together
    // weights as B operands: w1t[h][f], w2t[o][h] are N x K row-major
    for (uint32_t c = tid; c < NH * NF / 8; c += TC_FWD_THREADS) {
        const uint32_t r = c / (NF / 8), kc = c % (NF / 8);
        *reinterpret_cast<uint4 *>(tcs + TC_B1 + cm_off(r, kc * 8, NF)) =
            reinterpret_cast<const uint4 *>(w1t)[c];
    }
    for (uint32_t c = tid; c < NH * NH / 8; c += TC_FWD_THREADS) {
        const uint32_t r = c / (NH / 8), kc = c % (NH / 8);
        *reinterpret_cast<uint4 *>(tcs + TC_B2 + cm_off(r, kc * 8, NH)) =
            reinterpret_cast<const uint4 *>(w2t)[c];
    }
    for (uint32_t i = tid; i < NH; i += TC_FWD_THREADS) {
        vb1[i] = P[P_B1 + i];
        vb2[i] = P[P_B2 + i];
        vw3[i] = P[P_W3 + i];
    }
    const float b3 = P[P_B3];
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(tbase, TC_TMEM_COLS);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tbase;
    const uint32_t lane_addr = tm + (((warp & 3u) * 32u) << 16);   // this warp's TMEM lanes
    const uint32_t c0 = wg * (NH / 2);                 // this warpgroup's first column
    const uint32_t sbase = smem_u32(tcs);
    constexpr uint32_t IDESC = umma_idesc_bf16(TC_M, NH);
    uint32_t phase = 0;
    bool stuck = false;
    auto wait_mma = [&]() {
        for (uint32_t it = 0; !mbar_try_wait(bar, phase); it++)
            if (it >= TC_WAIT_POLLS) {
                stuck = true;
                break;
            }
        phase ^= 1u;
        tc_fence_after();
    };
    for (uint32_t rb = blockIdx.x * TC_M; rb < n; rb += gridDim.x * TC_M) {   // same trip count in every thread
        // X tile (rows past n are zero)
        for (uint32_t c = tid; c < TC_M * NF / 8; c += TC_FWD_THREADS) {
            const uint32_t r = c / (NF / 8), kc = c % (NF / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (rb + r < n) v = reinterpret_cast<const uint4 *>(X)[(size_t)(rb + r) * (NF / 8) + kc];
            *reinterpret_cast<uint4 *>(tcs + TC_A1 + cm_off(r, kc * 8, NF)) = v;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {                                  // layer 1: one K = 16 step
            umma_bf16(tm, umma_desc(sbase + TC_A1, 128, NF / 8 * 128), umma_desc(sbase + TC_B1, 128, NF / 8 * 128),
                      IDESC, 0);
            umma_commit(bar);
        }
        wait_mma();
        // layer-1 epilogue: bias, ReLU, BF16 -> A operand of layer 2
#pragma unroll
        for (uint32_t cc = 0; cc < NH / 64; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + col, v);
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                uint4 pk;
                uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
                for (uint32_t e = 0; e < 4; e++) {
                    const uint32_t h = col + q * 8 + 2 * e;
                    pw[e] = pack_bf16(fmaxf(v[q * 8 + 2 * e] + vb1[h], 0.f),
                                      fmaxf(v[q * 8 + 2 * e + 1] + vb1[h + 1], 0.f));
                }
                *reinterpret_cast<uint4 *>(tcs + TC_A2 + cm_off(row, col + q * 8, NH)) = pk;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {                                  // layer 2: K = 128 in 8 steps
#pragma unroll
            for (uint32_t s = 0; s < NH / 16; s++)
                umma_bf16(tm + NH, umma_desc(sbase + TC_A2 + s * 256, 128, NH / 8 * 128),
                          umma_desc(sbase + TC_B2 + s * 256, 128, NH / 8 * 128), IDESC, s);
            umma_commit(bar);
        }
        wait_mma();
        // layer-2 epilogue: bias, ReLU, dot with w3 over this half's columns
        float acc = 0.f;
#pragma unroll
        for (uint32_t cc = 0; cc < NH / 64; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + NH + col, v);
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) acc += fmaxf(v[j] + vb2[col + j], 0.f) * vw3[col + j];
        }
        if (wg == 1) half_sum[row] = acc;
        tc_fence_before();
        __syncthreads();                                 // the tiles and TMEM are free again
        tc_fence_after();
        if (wg == 0 && rb + row < n) y[rb + row] = b3 + acc + half_sum[row];
    }
    if (stuck) atomicOr(status, ST_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, TC_TMEM_COLS);
}

// ------------------------------------------------------------------ training on tcgen05

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Column sums of a warp's 32 x 32 block: lane L holds row L's values v[0..31];
// afterwards v[0] of lane j is the sum over the 32 rows of column j (each
// step halves the columns a lane keeps and adds its partner's share of them).
__device__ __forceinline__ float warp_column_sums(float (&v)[32], uint32_t lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & (uint32_t)s) != 0;
#pragma unroll
        for (int i = 0; i < s; i++) {
            const float send = upper ? v[i] : v[i + s];
            const float keep = upper ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, s);
        }
    }
    return v[0];
}

// shared-memory layout of the training kernel (bytes); operand tiles are
// K-major core-matrix tiles as in k_mlp_forward_tc
constexpr uint32_t TG_B1 = 0;                          // W1^T as B: N = 128 (h) x K = 16 (f)
constexpr uint32_t TG_B2 = TG_B1 + NH * NF * 2;        // W2^T as B: N = 128 (o) x K = 128 (h)
constexpr uint32_t TG_BW = TG_B2 + NH * NH * 2;        // W2 as B:   N = 128 (h) x K = 128 (o)
constexpr uint32_t TG_A1 = TG_BW + NH * NH * 2;        // X tile:    M = 128 (r) x K = 16 (f)
constexpr uint32_t TG_BX = TG_A1 + TC_M * NF * 2;      // X^T as B:  N = 16 (f) x K = 128 (r)
constexpr uint32_t TG_A2 = TG_BX + NF * TC_M * 2;      // h1 [r][h], then dZ2 [r][o]
constexpr uint32_t TG_A3 = TG_A2 + TC_M * NH * 2;      // h1^T [h][r], then dZ1^T [h][r]
constexpr uint32_t TG_BD = TG_A3 + NH * TC_M * 2;      // dZ2^T as B: N = 128 (o) x K = 128 (r)
constexpr uint32_t TG_VEC = TG_BD + NH * TC_M * 2;     // b1, b2, w3 (FP32)
constexpr uint32_t TG_XCH = TG_VEC + 3 * NH * 4;       // per row: second half's output sum, dy
constexpr uint32_t TG_BAR = TG_XCH + 2 * TC_M * 4;     // mbarrier, TMEM base address
constexpr uint32_t TG_SMEM = TG_BAR + 16;
// TMEM columns: z1 then dH1 [0, 128), z2 [128, 256), dW2 [256, 384), dW1^T [384, 400)
constexpr uint32_t TG_TMEM_COLS = 512;
static_assert(TG_SMEM <= 227u * 1024u, "training tiles exceed shared memory");

constexpr uint32_t TG_THREADS = 2 * TC_M;         // two warpgroups: column halves of each row

// Gradient of the mean squared error over rows [0, n) (same BF16 roundings
// as inference: weights and layer-1 activations; straight-through), 128 rows
// per tile on the tensor cores: forward z1 = X W1, z2 = h1 W2; backward
// dW2 = h1^T dZ2, dH1 = dZ2 W2^T, dW1 = X^T dZ1 with dZ2 and dZ1 rounded to
// BF16 as MMA operands (FP32 accumulation in TMEM across the block's tiles);
// the bias and w3 gradients and the loss are FP32 column sums.  Two
// warpgroups share every epilogue: warp w reads the TMEM lanes of warp
// w mod 4 (its rows), warpgroup 0 the columns 0-63 and warpgroup 1 the
// columns 64-127 of each accumulator.  Adds to G[] and *loss; *status gets
// ST_TIMEOUT if an MMA completion was not seen within the wait bound.  At
// most one block per SM (512 TMEM columns).
__global__ void __launch_bounds__(TG_THREADS, 1) k_mlp_grad_tc(
    const __nv_bfloat16 *__restrict__ X, const float *__restrict__ T, uint32_t n,
    const float *__restrict__ P, float *__restrict__ G, float *__restrict__ loss, uint32_t *status)
{
    extern __shared__ __align__(1024) uint8_t tgs[];
    float *vb1 = reinterpret_cast<float *>(tgs + TG_VEC), *vb2 = vb1 + NH, *vw3 = vb2 + NH;
    float *xch = reinterpret_cast<float *>(tgs + TG_XCH);       // per row: the other half's sum, then dy
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(tgs + TG_BAR);
    uint32_t *tbase = reinterpret_cast<uint32_t *>(tgs + TG_BAR + 8);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t r = tid & (TC_M - 1), wg = tid / TC_M;       // this thread's tile row and column half
    const uint32_t c0 = wg * (NH / 2);
    if (blockIdx.x * TC_M >= n) return;                // the whole block leaves together
    auto st_bf16 = [&](uint32_t off, float v) {
        *reinterpret_cast<__nv_bfloat16 *>(tgs + off) = __float2bfloat16_rn(v);
    };
    // weights, rounded to BF16, as B operands
    for (uint32_t i = tid; i < NF * NH; i += TG_THREADS) {   // (h, f) = W1[f][h]
        const uint32_t h = i / NF, f = i % NF;
        st_bf16(TG_B1 + cm_off(h, f, NF), P[P_W1 + f * NH + h]);
    }
    for (uint32_t i = tid; i < NH * NH; i += TG_THREADS) {   // W2[a][b]
        const uint32_t a = i / NH, b = i % NH;
        const float w = P[P_W2 + i];
        st_bf16(TG_B2 + cm_off(b, a, NH), w);                  // (o, h) = W2[h][o]
        st_bf16(TG_BW + cm_off(a, b, NH), w);                  // (h, o) = W2[h][o]
    }
    for (uint32_t i = tid; i < NH; i += TG_THREADS) {
        vb1[i] = P[P_B1 + i];
        vb2[i] = P[P_B2 + i];
        vw3[i] = P[P_W3 + i];
    }
    const float b3 = P[P_B3];
    const float inv_n = 1.0f / (float)n;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(tbase, TG_TMEM_COLS);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tbase;
    const uint32_t lane_addr = tm + (((warp & 3u) * 32u) << 16);
    const uint32_t sb = smem_u32(tgs);
    constexpr uint32_t ID_128 = umma_idesc_bf16(TC_M, NH), ID_16 = umma_idesc_bf16(TC_M, NF);
    constexpr uint32_t SBO16 = NF / 8 * 128, SBO128 = NH / 8 * 128;
    uint32_t phase = 0;
    bool stuck = false;
    auto wait_mma = [&]() {
        for (uint32_t it = 0; !mbar_try_wait(bar, phase); it++)
            if (it >= TC_WAIT_POLLS) {
                stuck = true;
                break;
            }
        phase ^= 1u;
        tc_fence_after();
    };
    auto sync_for_mma = [&]() {                          // generic smem writes -> MMA operands
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    };
    // column sums, lane j of a warp: columns c0 + 32 cc + j of its rows
    float acc_b1[2] = {0.f, 0.f}, acc_b2[2] = {0.f, 0.f}, acc_w3[2] = {0.f, 0.f};
    float acc_loss = 0.f, acc_b3 = 0.f;
    uint32_t first = 1;
    for (uint32_t rb = blockIdx.x * TC_M; rb < n; rb += gridDim.x * TC_M) {   // same trip count in every thread
        const bool valid = rb + r < n;
        // X tile as A (rows) and as B (transposed): warpgroup wg moves features 8 wg .. 8 wg + 7
        {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (valid) v = reinterpret_cast<const uint4 *>(X)[(size_t)(rb + r) * 2 + wg];
            *reinterpret_cast<uint4 *>(tgs + TG_A1 + cm_off(r, wg * 8, NF)) = v;
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (uint32_t f = 0; f < 8; f++)
                *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_BX + cm_off(wg * 8 + f, r, TC_M)) = e[f];
        }
        const float tgt = valid ? T[rb + r] : 0.f;
        sync_for_mma();
        if (tid == 0) {                                  // z1 = X W1
            umma_bf16(tm, umma_desc(sb + TG_A1, 128, SBO16), umma_desc(sb + TG_B1, 128, SBO16), ID_128, 0);
            umma_commit(bar);
        }
        wait_mma();
        // h1 = bf16(relu(z1 + b1)) -> A2 [r][h] and A3 [h][r]; keep its sign mask
        uint32_t m1[2];
#pragma unroll
        for (uint32_t cc = 0; cc < 2; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + col, v);
            m1[cc] = 0;
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                uint4 pk;
                uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
                for (uint32_t e = 0; e < 4; e++) {
                    const uint32_t j = q * 8 + 2 * e, h = col + j;
                    const __nv_bfloat162 hb = __floats2bfloat162_rn(fmaxf(v[j] + vb1[h], 0.f),
                                                                    fmaxf(v[j + 1] + vb1[h + 1], 0.f));
                    pw[e] = *reinterpret_cast<const uint32_t *>(&hb);
                    if (__bfloat162float(hb.x) > 0.f) m1[cc] |= 1u << j;
                    if (__bfloat162float(hb.y) > 0.f) m1[cc] |= 1u << (j + 1);
                    *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_A3 + cm_off(h, r, TC_M)) = hb.x;
                    *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_A3 + cm_off(h + 1, r, TC_M)) = hb.y;
                }
                *reinterpret_cast<uint4 *>(tgs + TG_A2 + cm_off(r, col + q * 8, NH)) = pk;
            }
        }
        sync_for_mma();
        if (tid == 0) {                                  // z2 = h1 W2
#pragma unroll
            for (uint32_t s = 0; s < NH / 16; s++)
                umma_bf16(tm + NH, umma_desc(sb + TG_A2 + s * 256, 128, SBO128),
                          umma_desc(sb + TG_B2 + s * 256, 128, SBO128), ID_128, s);
            umma_commit(bar);
        }
        wait_mma();
        // output: this half's share of w3 . relu(z2 + b2), the halves added
        // through shared memory; error and dy (rows past n contribute nothing)
        float yv = 0.f;
#pragma unroll
        for (uint32_t cc = 0; cc < 2; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + NH + col, v);
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) yv += fmaxf(v[j] + vb2[col + j], 0.f) * vw3[col + j];
        }
        if (wg == 1) xch[r] = yv;
        __syncthreads();
        if (wg == 0) {
            const float err = valid ? b3 + yv + xch[r] - tgt : 0.f;
            const float d = 2.f * err * inv_n;
            acc_loss += err * err;
            acc_b3 += d;
            xch[TC_M + r] = d;
        }
        __syncthreads();
        const float dy = xch[TC_M + r];
        // dZ2 = dy w3 [z2 + b2 > 0] -> A2 [r][o] (BF16) and BD [o][r]; w3 and b2 column sums
#pragma unroll
        for (uint32_t cc = 0; cc < 2; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32], gw[32];
            tmem_ld32(lane_addr + NH + col, v);
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) {
                const uint32_t o = col + j;
                const float z = v[j] + vb2[o];
                gw[j] = z > 0.f ? dy * z : 0.f;
                v[j] = z > 0.f ? dy * vw3[o] : 0.f;
            }
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                uint4 pk;
                uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
                for (uint32_t e = 0; e < 4; e++) {
                    const uint32_t j = q * 8 + 2 * e, o = col + j;
                    const __nv_bfloat162 db = __floats2bfloat162_rn(v[j], v[j + 1]);
                    pw[e] = *reinterpret_cast<const uint32_t *>(&db);
                    *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_BD + cm_off(o, r, TC_M)) = db.x;
                    *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_BD + cm_off(o + 1, r, TC_M)) = db.y;
                }
                *reinterpret_cast<uint4 *>(tgs + TG_A2 + cm_off(r, col + q * 8, NH)) = pk;
            }
            acc_w3[cc] += warp_column_sums(gw, lane);
            acc_b2[cc] += warp_column_sums(v, lane);
        }
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (uint32_t s = 0; s < TC_M / 16; s++)     // dW2 += h1^T dZ2 (K = rows)
                umma_bf16(tm + 2 * NH, umma_desc(sb + TG_A3 + s * 256, 128, SBO128),
                          umma_desc(sb + TG_BD + s * 256, 128, SBO128), ID_128, (s | (first ^ 1u)) != 0);
#pragma unroll
            for (uint32_t s = 0; s < NH / 16; s++)       // dH1 = dZ2 W2^T (K = o)
                umma_bf16(tm, umma_desc(sb + TG_A2 + s * 256, 128, SBO128),
                          umma_desc(sb + TG_BW + s * 256, 128, SBO128), ID_128, s);
            umma_commit(bar);
        }
        wait_mma();
        // dZ1 = dH1 [h1 > 0] -> A3 [h][r] (BF16); b1 column sums
#pragma unroll
        for (uint32_t cc = 0; cc < 2; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + col, v);
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) {
                v[j] = (m1[cc] >> j) & 1u ? v[j] : 0.f;
                *reinterpret_cast<__nv_bfloat16 *>(tgs + TG_A3 + cm_off(col + j, r, TC_M)) =
                    __float2bfloat16_rn(v[j]);
            }
            acc_b1[cc] += warp_column_sums(v, lane);
        }
        sync_for_mma();
        if (tid == 0) {                                  // dW1^T += dZ1^T X (K = rows)
#pragma unroll
            for (uint32_t s = 0; s < TC_M / 16; s++)
                umma_bf16(tm + 3 * NH, umma_desc(sb + TG_A3 + s * 256, 128, SBO128),
                          umma_desc(sb + TG_BX + s * 256, 128, SBO128), ID_16, (s | (first ^ 1u)) != 0);
            umma_commit(bar);
        }
        wait_mma();
        first = 0;
        tc_fence_before();
        __syncthreads();                                 // A1, BX, A2, A3, BD are free again
        tc_fence_after();
    }
    // dW2[h][o] is TMEM lane h, column 256 + o; dW1[f][h] lane h, column 384 + f
    {
        const uint32_t h = r;
#pragma unroll
        for (uint32_t cc = 0; cc < 2; cc++) {
            const uint32_t col = c0 + cc * 32;
            float v[32];
            tmem_ld32(lane_addr + 2 * NH + col, v);
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) atomicAdd(&G[P_W2 + h * NH + col + j], v[j]);
        }
        if (wg == 0) {
            float w[16];
            tmem_ld16(lane_addr + 3 * NH, w);
#pragma unroll
            for (uint32_t f = 0; f < NF; f++) atomicAdd(&G[P_W1 + f * NH + h], w[f]);
        }
    }
#pragma unroll
    for (uint32_t cc = 0; cc < 2; cc++) {                // lane j: column c0 + 32 cc + j
        atomicAdd(&G[P_B1 + c0 + cc * 32 + lane], acc_b1[cc]);
        atomicAdd(&G[P_B2 + c0 + cc * 32 + lane], acc_b2[cc]);
        atomicAdd(&G[P_W3 + c0 + cc * 32 + lane], acc_w3[cc]);
    }
    if (wg == 0) {
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            acc_loss += __shfl_xor_sync(FULL, acc_loss, d);
            acc_b3 += __shfl_xor_sync(FULL, acc_b3, d);
        }
        if (lane == 0) {
            atomicAdd(loss, acc_loss * inv_n);
            atomicAdd(&G[P_B3], acc_b3);
        }
    }
    if (stuck) atomicOr(status, ST_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, TG_TMEM_COLS);
}

// ------------------------------------------------------------------ optimiser

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

// Seeds are enumerated heaviest predicted first (longest processing time
// first): the launch's tail then holds light seeds, not a late hub whose
// subtree the idle warps must wait to be split off.  The order is by buckets
// of half a log2 unit of predicted cost; bucket 0 holds the heaviest.
constexpr uint32_t PICK_BUCKETS = 64;

__device__ __forceinline__ uint32_t cost_bucket(float log2_cycles)
{
    const float h = fminf(fmaxf(2.f * log2_cycles, 0.f), (float)(PICK_BUCKETS - 1));
    return PICK_BUCKETS - 1 - (uint32_t)h;
}

// The autotuner's margin trial.  A margin matters only for a seed whose
// model pick beats the paper's order by a predicted gain g = y0 - y_best in
// (0, m_max), m_max the largest candidate margin: outside it every candidate
// makes the same choice.  The candidate margins m_0 = 0 < m_1 < ... cut
// [0, m_max) into intervals [m_i, m_i+1); a seed whose gain falls in
// interval i takes the paper's order or the model's pick with equal odds
// (splitmix64 of seed index and round), slot 2 i + arm in its seed word and
// in mt.q_seeds, so each interval compares the two arms on a random half of
// the same batches' seeds.  Other seeds take the paper's order (g = 0) or
// the pick (g >= m_max) and slot MARGIN_SLOTS - 1.
struct MarginTrial {
    float m[MARGIN_SLOTS / 2];          // candidate margins, ascending, m[0] = 0
    uint32_t n;                         // candidates; 0: no trial
    uint32_t round;
    uint32_t *q_seeds;                  // [q][MARGIN_SLOTS]
};

// Per seed: the candidate order with the smallest predicted cost, but the
// paper's order (candidate 0) unless the best prediction beats it by at least
// the margin (log2 units; q_margin[q] for the seed's query q): the paper's
// order is the fallback.  During a margin trial (mt.n > 0) the seeds whose
// choice depends on the margin are split at random instead (MarginTrial).
__global__ void k_pick(const unsigned long long *seeds, const uint32_t *nseeds, uint32_t seed_cap,
                       const float *y, const float *q_margin, MarginTrial mt, float split_log2,
                       unsigned long long *picked, uint8_t *bucket, uint32_t *hist)
{
    __shared__ uint32_t sh[PICK_BUCKETS];
    for (uint32_t i = threadIdx.x; i < PICK_BUCKETS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t n = min(*nseeds, seed_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        uint32_t best = 0;
        const float y0 = y[(size_t)s * NCAND];
        float bv = y0;
        for (uint32_t k = 1; k < NCAND; k++) {
            const float v = y[(size_t)s * NCAND + k];
            if (v < bv) { bv = v; best = k; }
        }
        const unsigned long long sd = seeds[s];
        const uint32_t q = (uint32_t)(sd >> 8) & 0xffffu;
        uint32_t slot = MARGIN_SLOTS - 1;
        if (mt.n) {
            const float gain = y0 - bv;                  // >= 0; 0 when the paper's order is best
            uint32_t iv = mt.n;                          // interval of the gain
            if (best != 0)
                for (uint32_t i = 0; i + 1 < mt.n; i++)
                    if (gain >= mt.m[i] && gain < mt.m[i + 1]) iv = i;
            if (iv + 1 < mt.n) {
                unsigned long long z = ((unsigned long long)mt.round << 32) + s + 0x9E3779B97F4A7C15ull;
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                z ^= z >> 31;
                const uint32_t arm = (uint32_t)(z & 1u);   // 0: the paper's order, 1: the pick
                if (!arm) { best = 0; bv = y0; }
                slot = 2 * iv + arm;
                atomicAdd(&mt.q_seeds[q * MARGIN_SLOTS + slot], 1u);
            }
        } else if (bv > y0 - q_margin[q]) {
            best = 0;
            bv = y0;
        }
        unsigned long long w = (sd & ~(0xffull << 24)) | ((unsigned long long)best << 24) |
                               ((unsigned long long)slot << SEED_MARGIN_SHIFT);
        if (bv >= split_log2) w |= SEED_PRESPLIT;
        picked[s] = w;
        const uint32_t b = cost_bucket(bv);
        bucket[s] = (uint8_t)b;
        atomicAdd(&sh[b], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < PICK_BUCKETS; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Scatter the picked seeds into `seeds` by bucket, bucket 0 first (a counting
// sort; the order inside a bucket is arbitrary).  `cursor`: PICK_BUCKETS
// counters zeroed by the caller.  The positions taken in bucket b total
// hist[b], so every write lands in [0, n).  blockDim.x >= 32.
__global__ void k_seed_order(const unsigned long long *picked, const uint8_t *bucket, const uint32_t *nseeds,
                             uint32_t seed_cap, const uint32_t *hist, uint32_t *cursor,
                             unsigned long long *seeds)
{
    __shared__ uint32_t base[PICK_BUCKETS], cnt[PICK_BUCKETS], res[PICK_BUCKETS];
    static_assert(PICK_BUCKETS == 64, "two buckets per lane of one warp");
    if (threadIdx.x < 32) {                 // exclusive prefix of the bucket sizes
        const uint32_t b0 = 2 * threadIdx.x, v0 = hist[b0], v1 = hist[b0 + 1];
        uint32_t inc = v0 + v1;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(FULL, inc, o);
            if ((int)threadIdx.x >= o) inc += u;
        }
        base[b0] = inc - v0 - v1;
        base[b0 + 1] = inc - v1;
    }
    const uint32_t n = min(*nseeds, seed_cap);
    const uint32_t step = gridDim.x * blockDim.x;
    for (uint32_t t0 = blockIdx.x * blockDim.x; t0 < n; t0 += step) {     // uniform over the block
        for (uint32_t i = threadIdx.x; i < PICK_BUCKETS; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const uint32_t s = t0 + threadIdx.x;
        const bool in = s < n;
        const uint32_t b = in ? bucket[s] : 0u;
        const uint32_t r = in ? atomicAdd(&cnt[b], 1u) : 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < PICK_BUCKETS; i += blockDim.x)
            res[i] = cnt[i] ? atomicAdd(&cursor[i], cnt[i]) : 0u;
        __syncthreads();
        if (in) seeds[base[b] + res[b] + r] = picked[s];
        __syncthreads();
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
