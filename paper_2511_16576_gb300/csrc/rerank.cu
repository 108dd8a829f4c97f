// rerank.cu -- A7: learned reranker of bucket candidates (not in the paper).
//
// A small MLP maps features of a (query, candidate) pair to a predicted
// Jaccard similarity; candidates are then ordered by it (A6) so the exact
// refinement (A8) touches fewer of them.  Network 40 -> 64 -> 64 -> 1, ReLU,
// ReLU, sigmoid, mean squared error against the exact Jaccard.
//
// Features (bf16, padded to 48 columns; computed by the agreement kernel, A5):
//   0..31  group-match bits: bit j = all K/32 hashes of group j agree (and are
//          not the sentinel) -- the band-match pattern of a 32-band split;
//   32     agreement fraction c / K (Theorem 1 estimate of J);
//   33, 34 log2 of the query's and the candidate's area / 32;
//   35, 36 log2 of the query's and the candidate's vertex count / 16;
//   37, 38 fractions of hashes with h_k(q) < h_k(p) and h_k(q) > h_k(p): by the
//          min form of the hash their expectations are area(q \ p) / area(q u p)
//          and area(p \ q) / area(q u p), which, with the exact areas, sharpen
//          the overlap estimate where the two areas differ;
//   39     an upper bound of J: min(|q|, |p|, bounding-box overlap) over
//          |q| + |p| minus that minimum (a geometric prior the hashes lack).
//
// The forward pass (the scoring inside the query graph) runs on the
// fifth-generation tensor cores: tcgen05 MMAs from shared-memory operands into
// tensor-memory accumulators (mlp_tc_kernel, below).  Training runs its GEMMs
// with mma.sync m16n8k16 (bf16 operands, fp32 accumulation): one warp owns 16
// rows; the accumulator fragment of one layer is, element for element, the A
// fragment of the next, so activations stay in registers.  Training fuses
// forward and backward per 128-row chunk:
// activations and back-propagated gradients go to shared memory, weight
// gradients are tensor-core GEMMs over the chunk's rows (K = rows), kept in
// registers across chunks and added to global memory once per CTA.  Operand
// rounding points follow the fp64 reference exactly: weights, layer inputs and
// the back-propagated gradients feeding a GEMM are bf16; sums are fp32.
#include <cuda_bf16.h>

#include <algorithm>

#include "pmh_internal.cuh"

namespace {

constexpr int kIn = PMH_RERANK_IN;      // 40
constexpr int kInPad = 48;
constexpr int kH = PMH_RERANK_HIDDEN;   // 64
constexpr int kWarpsMlp = 8;
constexpr int kChunk = kWarpsMlp * 16;  // rows per CTA iteration
constexpr int XS = 56;                  // shared row strides (bf16), bank-conflict padding
constexpr int HS = 72;

// packed parameter / gradient layout
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + kH * kIn;
constexpr int OFF_W2 = OFF_B1 + kH;
constexpr int OFF_B2 = OFF_W2 + kH * kH;
constexpr int OFF_W3 = OFF_B2 + kH;
constexpr int OFF_B3 = OFF_W3 + kH;
constexpr int N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == PMH_RERANK_PARAMS, "packed layout");

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

struct MlpSmem {
    __nv_bfloat16 w1[kH][XS];   // [out][in]   B operand of layer 1
    __nv_bfloat16 w2[kH][HS];   // [out][in]   B operand of layer 2
    __nv_bfloat16 w2t[kH][HS];  // [in][out]   B operand of dh1 = d2 . W2
    __nv_bfloat16 w3[8][HS];    // row 0 = w3, rows 1..7 zero
    float b1[kH], b2[kH], w3f[kH], b3;
    __nv_bfloat16 x[kChunk][XS];
    __nv_bfloat16 h1[kChunk][HS];
    __nv_bfloat16 d2[kChunk][HS];
    __nv_bfloat16 d1[kChunk][HS];
    float g3[kChunk];
    float gb1[kH], gb2[kH], gw3[kH], gb3, loss;
};

// load the bf16 weights into shared memory (padding zeroed)
__device__ void load_weights(MlpSmem& s, const __nv_bfloat16* __restrict__ w1b,
                             const __nv_bfloat16* __restrict__ w2b,
                             const __nv_bfloat16* __restrict__ w3b, const float* __restrict__ master)
{
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int i = threadIdx.x; i < kH * XS; i += blockDim.x) {
        int o = i / XS, c = i % XS;
        s.w1[o][c] = c < kInPad ? w1b[o * kInPad + c] : zero;
    }
    for (int i = threadIdx.x; i < kH * HS; i += blockDim.x) {
        int o = i / HS, c = i % HS;
        s.w2[o][c] = c < kH ? w2b[o * kH + c] : zero;
        s.w2t[o][c] = c < kH ? w2b[c * kH + o] : zero;
    }
    for (int i = threadIdx.x; i < 8 * HS; i += blockDim.x) {
        int r = i / HS, c = i % HS;
        s.w3[r][c] = (r == 0 && c < kH) ? w3b[c] : zero;
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        s.b1[i] = master[OFF_B1 + i];
        s.b2[i] = master[OFF_B2 + i];
        s.w3f[i] = __bfloat162float(w3b[i]);
        s.gb1[i] = 0.f;
        s.gb2[i] = 0.f;
        s.gw3[i] = 0.f;
    }
    if (threadIdx.x == 0) {
        s.b3 = master[OFF_B3];
        s.gb3 = 0.f;
        s.loss = 0.f;
    }
}

// Training pass: forward + backward, accumulating the gradients of the mean
// squared error over n_total rows (the forward pass alone runs on tcgen05 below).
__global__ void __launch_bounds__(kWarpsMlp * 32, 1)
mlp_train_kernel(const __nv_bfloat16* __restrict__ feat, const float* __restrict__ label, int64_t n_rows,
                 int64_t n_total, const __nv_bfloat16* __restrict__ w1b,
                 const __nv_bfloat16* __restrict__ w2b, const __nv_bfloat16* __restrict__ w3b,
                 const float* __restrict__ master, float* __restrict__ grads, float* __restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    load_weights(s, w1b, w2b, w3b, master);
    __syncthreads();

    // weight-gradient accumulators of this warp, kept across chunks:
    // gW2 slice: out units 16*(wid/2).., in units 32*(wid%2).. (4 n-tiles);
    // gW1 slice: out units 16*(wid/2).., in units 24*(wid%2).. (3 n-tiles)
    float acc_w2[4][4] = {};
    float acc_w1[3][4] = {};
    const float inv_n = 1.f / (float)(n_total > 1 ? n_total : 1);

    for (int64_t base = (int64_t)blockIdx.x * kChunk; base < n_rows; base += (int64_t)gridDim.x * kChunk) {
        // stage the chunk's features (rows past n_rows are zero)
        for (int i = threadIdx.x; i < kChunk * (kInPad / 2); i += blockDim.x) {
            int r = i / (kInPad / 2), c2 = i % (kInPad / 2);
            uint32_t v = 0;
            if (base + r < n_rows) v = ld32(feat + (base + r) * kInPad + 2 * c2);
            *reinterpret_cast<uint32_t*>(&s.x[r][2 * c2]) = v;
        }
        __syncthreads();
        const int r0 = wid * 16;  // this warp's rows within the chunk

        // ---- layer 1: [16 x 48] x [48 x 64]
        float acc1[8][4] = {};
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            uint32_t a[4] = {ld32(&s.x[r0 + g][16 * kk + 2 * t]), ld32(&s.x[r0 + g + 8][16 * kk + 2 * t]),
                             ld32(&s.x[r0 + g][16 * kk + 2 * t + 8]),
                             ld32(&s.x[r0 + g + 8][16 * kk + 2 * t + 8])};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2] = {ld32(&s.w1[nt * 8 + g][16 * kk + 2 * t]),
                                 ld32(&s.w1[nt * 8 + g][16 * kk + 2 * t + 8])};
                mma_bf16(acc1[nt], a, b);
            }
        }
        uint32_t a2f[4][4];
        uint32_t mask1 = 0;  // bit (nt*4 + i): z1 > 0 for element i of n-tile nt
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float h[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float z = acc1[nt][i] + s.b1[nt * 8 + 2 * t + (i & 1)];
                mask1 |= (uint32_t)(z > 0.f) << (nt * 4 + i);
                h[i] = z > 0.f ? z : 0.f;
            }
            uint32_t lo = pack2(h[0], h[1]), hi = pack2(h[2], h[3]);
            a2f[nt >> 1][(nt & 1) * 2 + 0] = lo;
            a2f[nt >> 1][(nt & 1) * 2 + 1] = hi;
            *reinterpret_cast<uint32_t*>(&s.h1[r0 + g][nt * 8 + 2 * t]) = lo;
            *reinterpret_cast<uint32_t*>(&s.h1[r0 + g + 8][nt * 8 + 2 * t]) = hi;
        }
        // ---- layer 2: [16 x 64] x [64 x 64]
        float acc2[8][4] = {};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2] = {ld32(&s.w2[nt * 8 + g][16 * kk + 2 * t]),
                                 ld32(&s.w2[nt * 8 + g][16 * kk + 2 * t + 8])};
                mma_bf16(acc2[nt], a2f[kk], b);
            }
        }
        uint32_t a3f[4][4];
        uint32_t mask2 = 0;
        float h2v[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float z = acc2[nt][i] + s.b2[nt * 8 + 2 * t + (i & 1)];
                mask2 |= (uint32_t)(z > 0.f) << (nt * 4 + i);
                h2v[nt][i] = bfr(z > 0.f ? z : 0.f);
            }
            uint32_t lo = pack2(h2v[nt][0], h2v[nt][1]), hi = pack2(h2v[nt][2], h2v[nt][3]);
            a3f[nt >> 1][(nt & 1) * 2 + 0] = lo;
            a3f[nt >> 1][(nt & 1) * 2 + 1] = hi;
        }
        // ---- layer 3: [16 x 64] x [64 x 8] (column 0 = w3)
        float acc3[4] = {};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t b[2] = {ld32(&s.w3[g][16 * kk + 2 * t]), ld32(&s.w3[g][16 * kk + 2 * t + 8])};
            mma_bf16(acc3, a3f[kk], b);
        }
        // rows r0+g (acc3[0]) and r0+g+8 (acc3[2]) live in lanes with t == 0
        const int64_t rowA = base + r0 + g, rowB = rowA + 8;
        float pA = 1.f / (1.f + expf(-(acc3[0] + s.b3)));
        float pB = 1.f / (1.f + expf(-(acc3[2] + s.b3)));
        // ---- backward
        if (t == 0) {
            float gA = 0.f, gB = 0.f, l = 0.f;
            if (rowA < n_rows) {
                float err = pA - label[rowA];
                l += err * err;
                gA = 2.f * err * inv_n * pA * (1.f - pA);
            }
            if (rowB < n_rows) {
                float err = pB - label[rowB];
                l += err * err;
                gB = 2.f * err * inv_n * pB * (1.f - pB);
            }
            s.g3[r0 + g] = gA;
            s.g3[r0 + g + 8] = gB;
            atomicAdd(&s.loss, l);
            atomicAdd(&s.gb3, gA + gB);
        }
        __syncwarp();
        const float g3A = s.g3[r0 + g], g3B = s.g3[r0 + g + 8];
        const float g3rA = bfr(g3A), g3rB = bfr(g3B);
        // d2 = bf16(relu'(z2) * w3 * g3r); gb2 += relu'(z2) * w3 * g3r; gw3 += g3r * h2
        uint32_t a4f[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4], gw[2], gb[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = nt * 8 + 2 * t + c;
                const float w3 = s.w3f[col];
                const bool mA = (mask2 >> (nt * 4 + c)) & 1u, mB = (mask2 >> (nt * 4 + 2 + c)) & 1u;
                d[c] = mA ? w3 * g3rA : 0.f;
                d[2 + c] = mB ? w3 * g3rB : 0.f;
                gb[c] = d[c] + d[2 + c];
                gw[c] = g3rA * h2v[nt][c] + g3rB * h2v[nt][2 + c];
            }
            // reduce over the 8 row groups g (lanes with equal t)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    gb[c] += __shfl_xor_sync(0xffffffffu, gb[c], o);
                    gw[c] += __shfl_xor_sync(0xffffffffu, gw[c], o);
                }
            }
            if (g == 0) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    atomicAdd(&s.gb2[nt * 8 + 2 * t + c], gb[c]);
                    atomicAdd(&s.gw3[nt * 8 + 2 * t + c], gw[c]);
                }
            }
            uint32_t lo = pack2(d[0], d[1]), hi = pack2(d[2], d[3]);
            a4f[nt >> 1][(nt & 1) * 2 + 0] = lo;
            a4f[nt >> 1][(nt & 1) * 2 + 1] = hi;
            *reinterpret_cast<uint32_t*>(&s.d2[r0 + g][nt * 8 + 2 * t]) = lo;
            *reinterpret_cast<uint32_t*>(&s.d2[r0 + g + 8][nt * 8 + 2 * t]) = hi;
        }
        // dh1 = d2 . W2 : [16 x 64 out] x [64 out x 64 in]
        float acc4[8][4] = {};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2] = {ld32(&s.w2t[nt * 8 + g][16 * kk + 2 * t]),
                                 ld32(&s.w2t[nt * 8 + g][16 * kk + 2 * t + 8])};
                mma_bf16(acc4[nt], a4f[kk], b);
            }
        }
        // d1 = relu'(z1) * dh1; gb1 += d1; d1 (bf16) to shared memory
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4], gb[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) d[i] = ((mask1 >> (nt * 4 + i)) & 1u) ? acc4[nt][i] : 0.f;
            gb[0] = d[0] + d[2];
            gb[1] = d[1] + d[3];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) gb[c] += __shfl_xor_sync(0xffffffffu, gb[c], o);
            if (g == 0) {
                atomicAdd(&s.gb1[nt * 8 + 2 * t], gb[0]);
                atomicAdd(&s.gb1[nt * 8 + 2 * t + 1], gb[1]);
            }
            *reinterpret_cast<uint32_t*>(&s.d1[r0 + g][nt * 8 + 2 * t]) = pack2(d[0], d[1]);
            *reinterpret_cast<uint32_t*>(&s.d1[r0 + g + 8][nt * 8 + 2 * t]) = pack2(d[2], d[3]);
        }
        __syncthreads();
        // weight gradients over the chunk's 128 rows (K = rows)
        const int m0 = 16 * (wid >> 1);
#pragma unroll
        for (int kk = 0; kk < kChunk / 16; ++kk) {
            const int k0 = 16 * kk;
            // A[m = out][k = row] = d2[row][out]
            uint32_t a[4] = {pack_raw(s.d2[k0 + 2 * t][m0 + g], s.d2[k0 + 2 * t + 1][m0 + g]),
                             pack_raw(s.d2[k0 + 2 * t][m0 + g + 8], s.d2[k0 + 2 * t + 1][m0 + g + 8]),
                             pack_raw(s.d2[k0 + 2 * t + 8][m0 + g], s.d2[k0 + 2 * t + 9][m0 + g]),
                             pack_raw(s.d2[k0 + 2 * t + 8][m0 + g + 8], s.d2[k0 + 2 * t + 9][m0 + g + 8])};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n0 = 32 * (wid & 1) + 8 * j;
                // B[k = row][n = in] = h1[row][in]
                uint32_t b[2] = {pack_raw(s.h1[k0 + 2 * t][n0 + g], s.h1[k0 + 2 * t + 1][n0 + g]),
                                 pack_raw(s.h1[k0 + 2 * t + 8][n0 + g], s.h1[k0 + 2 * t + 9][n0 + g])};
                mma_bf16(acc_w2[j], a, b);
            }
            uint32_t a1[4] = {pack_raw(s.d1[k0 + 2 * t][m0 + g], s.d1[k0 + 2 * t + 1][m0 + g]),
                              pack_raw(s.d1[k0 + 2 * t][m0 + g + 8], s.d1[k0 + 2 * t + 1][m0 + g + 8]),
                              pack_raw(s.d1[k0 + 2 * t + 8][m0 + g], s.d1[k0 + 2 * t + 9][m0 + g]),
                              pack_raw(s.d1[k0 + 2 * t + 8][m0 + g + 8], s.d1[k0 + 2 * t + 9][m0 + g + 8])};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int n0 = 24 * (wid & 1) + 8 * j;
                uint32_t b[2] = {pack_raw(s.x[k0 + 2 * t][n0 + g], s.x[k0 + 2 * t + 1][n0 + g]),
                                 pack_raw(s.x[k0 + 2 * t + 8][n0 + g], s.x[k0 + 2 * t + 9][n0 + g])};
                mma_bf16(acc_w1[j], a1, b);
            }
        }
        __syncthreads();
    }
    // flush: this warp's weight-gradient slices and the CTA's small partials
    const int m0 = 16 * (wid >> 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n0 = 32 * (wid & 1) + 8 * j;
        atomicAdd(&grads[OFF_W2 + (m0 + g) * kH + n0 + 2 * t], acc_w2[j][0]);
        atomicAdd(&grads[OFF_W2 + (m0 + g) * kH + n0 + 2 * t + 1], acc_w2[j][1]);
        atomicAdd(&grads[OFF_W2 + (m0 + g + 8) * kH + n0 + 2 * t], acc_w2[j][2]);
        atomicAdd(&grads[OFF_W2 + (m0 + g + 8) * kH + n0 + 2 * t + 1], acc_w2[j][3]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int n0 = 24 * (wid & 1) + 8 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = m0 + g + (i >= 2 ? 8 : 0), c = n0 + 2 * t + (i & 1);
            if (c < kIn) atomicAdd(&grads[OFF_W1 + o * kIn + c], acc_w1[j][i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        atomicAdd(&grads[OFF_B1 + i], s.gb1[i]);
        atomicAdd(&grads[OFF_B2 + i], s.gb2[i]);
        atomicAdd(&grads[OFF_W3 + i], s.gw3[i]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&grads[OFF_B3], s.gb3);
        atomicAdd(loss_out, s.loss * inv_n);
    }
}

// Adam on the fp32 master weights (the bf16 operand copies are refreshed after it)
__global__ void adam_kernel(float* __restrict__ master, float* __restrict__ m1,
                            float* __restrict__ m2, const float* __restrict__ grads, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_PARAMS; i += gridDim.x * blockDim.x) {
        float gr = grads[i];
        float a = beta1 * m1[i] + (1.f - beta1) * gr;
        float b = beta2 * m2[i] + (1.f - beta2) * gr * gr;
        m1[i] = a;
        m2[i] = b;
        float w = master[i] - lr * (a / bc1) / (sqrtf(b / bc2) + eps);
        master[i] = w;
    }
}

__global__ void refresh_bf16_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ w1b,
                                    __nv_bfloat16* __restrict__ w2b, __nv_bfloat16* __restrict__ w3b)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH * kInPad; i += gridDim.x * blockDim.x) {
        int o = i / kInPad, c = i % kInPad;
        w1b[i] = __float2bfloat16_rn(c < kIn ? master[OFF_W1 + o * kIn + c] : 0.f);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH * kH; i += gridDim.x * blockDim.x)
        w2b[i] = __float2bfloat16_rn(master[OFF_W2 + i]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH; i += gridDim.x * blockDim.x)
        w3b[i] = __float2bfloat16_rn(master[OFF_W3 + i]);
}

// ---------------------------------------------------------------------------
// Forward pass on the fifth-generation tensor cores (tcgen05, one CTA, no
// cluster): tiles of 128 rows; layer 1 is [128 x 48] x [48 x 64] and layer 2
// [128 x 64] x [64 x 64], each a chain of M=128, N=64, K=16 bf16 MMAs issued by
// one thread with fp32 accumulators in tensor memory (columns 0..63 and
// 64..127); the operands sit in shared memory in the canonical K-major layout
// without swizzle (core matrices of 8 rows x 16 bytes; the 16-byte rows of one
// core matrix are consecutive, core matrices adjacent in K are 128 bytes apart,
// groups of 8 rows are K * 16 bytes apart).  Thread 32w + l owns row 32w + l of
// the tile (tensor-memory lane 32w + l, which warp w may read): it adds the
// bias, applies ReLU and rounds to bf16 after each layer, exactly where the
// fp64 reference rounds, and computes layer 3 (64 -> 1) as a dot product.
// Every wait on the tensor cores is bounded: a wait that runs out sets `err`
// bit 16, the CTA stops, frees its tensor memory and returns.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kTcCols = 128;  // tensor-memory columns: two 64-column fp32 accumulators
constexpr int kTcErr = 16;

struct TcSmem {
    __nv_bfloat16 x[kTcRows * kInPad];  // the tile's features (canonical layout)
    __nv_bfloat16 h1[kTcRows * kH];     // layer-1 activations
    __nv_bfloat16 w1[kH * kInPad];      // W1 [out][in] (B operand, K-major)
    __nv_bfloat16 w2[kH * kH];          // W2 [out][in]
    float b1[kH], b2[kH], w3[kH], b3;
    unsigned long long mbar;
    uint32_t tmem;
    int stop;
};

// element offset of (row r, column k) in the canonical layout of a matrix with kd columns
__device__ __forceinline__ int canon(int r, int k, int kd)
{
    return (r >> 3) * (kd * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: fp32 accumulator, bf16 A and B, both K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* mbar)
{
    const uint32_t m = (uint32_t)__cvta_generic_to_shared(mbar);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(m)
                 : "memory");
}

// bounded wait for the phase of parity `phase` of the barrier; false if it ran out
__device__ __forceinline__ bool tc_wait(unsigned long long* mbar, uint32_t phase)
{
    const uint32_t m = (uint32_t)__cvta_generic_to_shared(mbar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(m), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// weights into shared memory, the barrier, the tensor-memory allocation
__device__ uint32_t tc_setup(TcSmem& s, const __nv_bfloat16* __restrict__ w1b,
                             const __nv_bfloat16* __restrict__ w2b, const __nv_bfloat16* __restrict__ w3b,
                             const float* __restrict__ master)
{
    const int tid = threadIdx.x, wid = tid >> 5;
    // eight consecutive inputs of an output row are 16 contiguous bytes on both sides
    for (int i = tid; i < kH * kInPad / 8; i += kTcThreads) {
        const int o = i / (kInPad / 8), c = 8 * (i % (kInPad / 8));
        *reinterpret_cast<uint4*>(s.w1 + canon(o, c, kInPad)) =
            __ldg(reinterpret_cast<const uint4*>(w1b + o * kInPad + c));
    }
    for (int i = tid; i < kH * kH / 8; i += kTcThreads) {
        const int o = i / (kH / 8), c = 8 * (i % (kH / 8));
        *reinterpret_cast<uint4*>(s.w2 + canon(o, c, kH)) = __ldg(reinterpret_cast<const uint4*>(w2b + o * kH + c));
    }
    for (int i = tid; i < kH; i += kTcThreads) {
        s.b1[i] = master[OFF_B1 + i];
        s.b2[i] = master[OFF_B2 + i];
        s.w3[i] = __bfloat162float(w3b[i]);
    }
    if (tid == 0) {
        s.b3 = master[OFF_B3];
        s.stop = 0;
        const uint32_t m = (uint32_t)__cvta_generic_to_shared(&s.mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (wid == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s.tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return s.tmem;
}

// The network on the tile's features in s.x (written by the CTA's threads just
// before): thread t returns the predicted Jaccard of row t.  False when a wait on
// the tensor cores ran out (s.stop set; the caller leaves its loop).
__device__ bool tc_tile(TcSmem& s, uint32_t tmem, uint32_t& phase, float& out)
{
    const int tid = threadIdx.x, wid = tid >> 5;
    const uint32_t lane_base = (uint32_t)(32 * wid) << 16;  // this warp's tensor-memory lanes
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 1: three K = 16 steps (two core matrices each, 128 elements apart) into
    // columns 0..63
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kInPad / 16; ++kk)
            tc_mma(tmem, tc_desc(s.x + 128 * kk, 128, kInPad * 16), tc_desc(s.w1 + 128 * kk, 128, kInPad * 16),
                   kk > 0);
        tc_commit(&s.mbar);
    }
    if (!tc_wait(&s.mbar, phase)) s.stop = 1;
    phase ^= 1u;
    tc_fence_after();
    __syncthreads();
    if (s.stop) return false;
    // epilogue 1: bias, ReLU, bf16, into the canonical layout of layer 2's A operand
    const int row = tid;
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
        float z[16];
        tc_ld16(tmem + lane_base + (uint32_t)c0, z);
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float a = z[j + 2 * u] + s.b1[c0 + j + 2 * u];
                const float b = z[j + 2 * u + 1] + s.b1[c0 + j + 2 * u + 1];
                pk[u] = pack2(a > 0.f ? a : 0.f, b > 0.f ? b : 0.f);
            }
            *reinterpret_cast<uint4*>(s.h1 + canon(row, c0 + j, kH)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 2: four K = 16 steps into columns 64..127
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kH / 16; ++kk)
            tc_mma(tmem + 64, tc_desc(s.h1 + 128 * kk, 128, kH * 16), tc_desc(s.w2 + 128 * kk, 128, kH * 16),
                   kk > 0);
        tc_commit(&s.mbar);
    }
    if (!tc_wait(&s.mbar, phase)) s.stop = 1;
    phase ^= 1u;
    tc_fence_after();
    __syncthreads();
    if (s.stop) return false;
    // epilogue 2: bias, ReLU, bf16 rounding, layer 3 and the sigmoid
    float acc = 0.f;
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
        float z[16];
        tc_ld16(tmem + lane_base + 64u + (uint32_t)c0, z);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float v = z[j] + s.b2[c0 + j];
            acc += bfr(v > 0.f ? v : 0.f) * s.w3[c0 + j];
        }
    }
    out = 1.f / (1.f + expf(-(acc + s.b3)));
    tc_fence_before();
    return true;
}

// the tensor memory back; a wait that ran out reports error bit 16
__device__ void tc_teardown(TcSmem& s, uint32_t tmem, int* err)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols)
                     : "memory");
    if (threadIdx.x == 0 && s.stop && err) atomicOr(err, kTcErr);
}

__global__ void __launch_bounds__(kTcThreads, 1)
mlp_tc_kernel(const __nv_bfloat16* __restrict__ feat, int64_t n_rows, const __nv_bfloat16* __restrict__ w1b,
              const __nv_bfloat16* __restrict__ w2b, const __nv_bfloat16* __restrict__ w3b,
              const float* __restrict__ master, float* __restrict__ score, int* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const uint32_t tmem = tc_setup(s, w1b, w2b, w3b, master);
    uint32_t phase = 0;
    for (int64_t base = (int64_t)blockIdx.x * kTcRows; base < n_rows; base += (int64_t)gridDim.x * kTcRows) {
        // the tile's features (16-byte chunks; rows past n_rows are zero)
        for (int i = tid; i < kTcRows * (kInPad / 8); i += kTcThreads) {
            const int r = i / (kInPad / 8), kc = i % (kInPad / 8);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (base + r < n_rows) v = *reinterpret_cast<const uint4*>(feat + (base + r) * kInPad + 8 * kc);
            *reinterpret_cast<uint4*>(s.x + canon(r, 8 * kc, kInPad)) = v;
        }
        float y;
        if (!tc_tile(s, tmem, phase, y)) break;
        if (base + tid < n_rows) score[base + tid] = y;
    }
    tc_teardown(s, tmem, err);
}

// ---------------------------------------------------------------------------
// Learned selection in one launch (the query graph's A7 and final A6 step).  A
// CTA takes 128 shortlist rows at a time -- 128 / S queries of S rows (the
// top-S by agreement count, ids [Q][S] and counts n[Q]) -- and
//  1. computes their feature rows straight into the tile's shared-memory
//     operand: each lane reads its row's id and polygon inputs, then each warp
//     compares eight pairs at a time (eight 16-byte loads of candidate hashes in
//     flight per lane) and takes the values from pmh_feature_values, as the
//     agreement kernel does;
//  2. scores them with the network on the tensor cores (tc_tile);
//  3. ranks each query's S scores (key = ~orderable(score) << 32 | id, as the
//     top-m kernel orders them) and writes the first m ids, -1 padded, and
//     min(m, n) -- the list the separate feature, forward and top-m launches give.
// Queries at or past *d_n, or all of them after a failed validation, get empty
// lists.  Needs K % 32 == 0 and S in {4, 8, .., 128} dividing 128.
// ---------------------------------------------------------------------------
constexpr int kSelPairs = 8;  // pairs compared at a time by a warp

// orderable float bits: larger float -> larger unsigned (the top-m kernel's order)
__device__ __forceinline__ uint32_t f2ord_sel(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

struct SelSmem {
    TcSmem tc;
    uint32_t eq[kTcThreads / 32][kSelPairs][4096 / 32];  // equality words, K <= 4096
    FeatPair fp[kTcThreads / 32][32];                     // each warp's rows' polygon inputs
    float score[kTcRows];
};

template <bool kOneQuery>  // S % kSelPairs == 0: the pairs compared together share their query
__global__ void __launch_bounds__(kTcThreads, 1)
rerank_select_kernel(const uint32_t* __restrict__ qh, const uint32_t* __restrict__ ph,
                     const int32_t* __restrict__ sl_ids, const int32_t* __restrict__ sl_n, int64_t Q,
                     const int64_t* __restrict__ d_n, int S, int m, int K, uint32_t T, FeatSrc qf, FeatSrc pf,
                     const __nv_bfloat16* __restrict__ w1b, const __nv_bfloat16* __restrict__ w2b,
                     const __nv_bfloat16* __restrict__ w3b, const float* __restrict__ master,
                     int32_t* __restrict__ out_ids, int32_t* __restrict__ out_n, const int* __restrict__ d_flags,
                     int* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SelSmem& ss = *reinterpret_cast<SelSmem*>(smem_raw);
    TcSmem& s = ss.tc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t tmem = tc_setup(s, w1b, w2b, w3b, master);
    const bool failed = d_flags && *d_flags;
    const int64_t live = failed ? 0 : (d_n ? min(Q, *d_n) : Q);
    const int G = kTcRows / S;  // queries per tile
    const int64_t tiles = (Q + G - 1) / G;
    const int K4 = K / 4;
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q0 = tile * G;
        // 1. feature rows 32 * wid .. 32 * wid + 31: each lane first reads its own row's
        //    candidate id and polygon inputs (one round of loads for the warp's rows), then
        //    the warp compares the rows' hashes eight pairs at a time
        const int rl = 32 * wid + lane;
        const int64_t ql = q0 + rl / S;
        const int nql = ql < live ? sl_n[ql] : 0;
        const bool okl = rl % S < nql;
        const int32_t pl = okl ? sl_ids[ql * S + rl % S] : 0;
        if (okl) ss.fp[wid][lane] = pmh_feat_pair(qf, pf, ql, pl);
        __syncwarp();
        for (int j0 = 0; j0 < 32; j0 += kSelPairs) {
            int64_t q[kSelPairs], p[kSelPairs];
            bool ok[kSelPairs];
#pragma unroll
            for (int t = 0; t < kSelPairs; ++t) {
                q[t] = q0 + (32 * wid + j0 + t) / S;
                p[t] = __shfl_sync(0xffffffffu, pl, j0 + t);
                ok[t] = __shfl_sync(0xffffffffu, (int)okl, j0 + t) != 0;
            }
            int c[kSelPairs], lt[kSelPairs], gt[kSelPairs];
            bool grp[kSelPairs];  // K = 128: lane l's four hashes (group l) all equal
#pragma unroll
            for (int t = 0; t < kSelPairs; ++t) {
                c[t] = lt[t] = gt[t] = 0;
                grp[t] = false;
            }
            if (__any_sync(0xffffffffu, okl && lane >= j0 && lane < j0 + kSelPairs)) {
                for (int base = 0; base < K4; base += 32) {
                    const int i = base + lane;
                    constexpr int kU = kOneQuery ? 1 : kSelPairs;  // query rows read
                    uint4 u[kU], v[kSelPairs];
#pragma unroll
                    for (int t = 0; t < kU; ++t) {
                        u[t] = make_uint4(0u, 0u, 0u, 0u);
                        if ((kOneQuery || ok[t]) && i < K4) u[t] = __ldg(reinterpret_cast<const uint4*>(qh + q[t] * K) + i);
                    }
#pragma unroll
                    for (int t = 0; t < kSelPairs; ++t) {
                        v[t] = make_uint4(0u, 0u, 0u, 0u);
                        if (ok[t] && i < K4) v[t] = __ldg(reinterpret_cast<const uint4*>(ph + p[t] * K) + i);
                    }
#pragma unroll
                    for (int t = 0; t < kSelPairs; ++t) {
                        const uint4 a = u[kOneQuery ? 0 : t], b = v[t];
                        unsigned bits = 0;
                        if (i < K4) {
                            bits = (unsigned)((a.x == b.x) & (a.x != T)) | ((unsigned)((a.y == b.y) & (a.y != T)) << 1) |
                                   ((unsigned)((a.z == b.z) & (a.z != T)) << 2) |
                                   ((unsigned)((a.w == b.w) & (a.w != T)) << 3);
                            lt[t] += (a.x < b.x) + (a.y < b.y) + (a.z < b.z) + (a.w < b.w);
                            gt[t] += (a.x > b.x) + (a.y > b.y) + (a.z > b.z) + (a.w > b.w);
                        }
                        c[t] += __popc(bits);
                        grp[t] = bits == 0xFu;
                        if (K != 128) {
                            // hash 4i+e is bit (4i+e) % 32 of word i / 8: OR eight lanes' nibbles
                            unsigned w0 = bits << ((lane & 7) * 4);
                            w0 |= __shfl_xor_sync(0xffffffffu, w0, 1);
                            w0 |= __shfl_xor_sync(0xffffffffu, w0, 2);
                            w0 |= __shfl_xor_sync(0xffffffffu, w0, 4);
                            if ((lane & 7) == 0 && i < K4) ss.eq[wid][t][i >> 3] = w0;
                        }
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kSelPairs; ++t) {
                const int r = 32 * wid + j0 + t;
                float lo = 0.f, hi = 0.f;
                if (ok[t]) {  // warp-uniform
                    int ct, lt_t, gt_t;
                    if (K < 1024) {  // the three counts in one sum (10 bits each)
                        const int sum = __reduce_add_sync(0xffffffffu, c[t] | (lt[t] << 10) | (gt[t] << 20));
                        ct = sum & 1023;
                        lt_t = (sum >> 10) & 1023;
                        gt_t = sum >> 20;
                    } else {
                        ct = __reduce_add_sync(0xffffffffu, c[t]);
                        lt_t = __reduce_add_sync(0xffffffffu, lt[t]);
                        gt_t = __reduce_add_sync(0xffffffffu, gt[t]);
                    }
                    if (K == 128) {
                        lo = grp[t] ? 1.f : 0.f;
                        hi = pmh_feature_col(lane, K, ct, lt_t, gt_t, ss.fp[wid][j0 + t]);
                    } else {
                        pmh_feature_values(ss.eq[wid][t], K, ct, lt_t, gt_t, ss.fp[wid][j0 + t], lane, lo, hi);
                    }
                }
                s.x[canon(r, lane, kInPad)] = __float2bfloat16_rn(lo);
                if (lane < 16) s.x[canon(r, 32 + lane, kInPad)] = __float2bfloat16_rn(hi);
            }
            __syncwarp();
        }
        // 2. the network
        float y;
        if (!tc_tile(s, tmem, phase, y)) break;
        ss.score[tid] = y;
        __syncthreads();
        // 3. each query's top m by (score desc, id asc): a pair's rank is the number of
        //    the query's keys below its own (ids within a list are distinct)
        for (int gq = wid; gq < G; gq += kTcThreads / 32) {
            const int64_t q = q0 + gq;
            if (q >= Q) continue;
            const int nq = q < live ? sl_n[q] : 0;
            const int kept = min(m, nq);
            const float* sc = ss.score + gq * S;
            const int32_t* ids = sl_ids + q * S;
            for (int i = lane; i < nq; i += 32) {
                const uint64_t ki = ((uint64_t)~f2ord_sel(sc[i]) << 32) | (uint32_t)ids[i];
                int rank = 0;
                for (int j = 0; j < nq; ++j)
                    rank += (((uint64_t)~f2ord_sel(sc[j]) << 32) | (uint32_t)ids[j]) < ki;
                if (rank < m) out_ids[q * m + rank] = ids[i];
            }
            for (int i = kept + lane; i < m; i += 32) out_ids[q * m + i] = -1;
            if (lane == 0) out_n[q] = kept;
        }
        __syncthreads();
    }
    tc_teardown(s, tmem, err);
}

}  // namespace

struct pmh_rerank_s {
    pmh_ctx ctx = nullptr;
    int device = 0;
    float* master = nullptr;  // packed fp32 weights
    float* m1 = nullptr;      // Adam moments
    float* m2 = nullptr;
    float* grads = nullptr;
    float* loss = nullptr;
    __nv_bfloat16* w1b = nullptr;  // [64][48] bf16 operand copies
    __nv_bfloat16* w2b = nullptr;  // [64][64]
    __nv_bfloat16* w3b = nullptr;  // [64]
    int* err = nullptr;            // tensor-core wait status of the public forward call
    int64_t steps = 0;
};

extern "C" int pmh_rerank_destroy(pmh_rerank r)
{
    if (!r) return PMH_OK;
    cudaSetDevice(r->device);
    cudaDeviceSynchronize();
    void* bufs[] = {r->master, r->m1, r->m2, r->grads, r->loss, r->w1b, r->w2b, r->w3b, r->err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete r;
    return PMH_OK;
}

extern "C" int pmh_rerank_create(pmh_ctx ctx, pmh_rerank* out)
{
    if (!out) return pmh_set_error(PMH_ERR_ARG, "null out");
    *out = nullptr;
    PMH_TRY(pmh_check_device(ctx));
    pmh_rerank r = new pmh_rerank_s();
    r->ctx = ctx;
    r->device = ctx->device;
    bool ok = cudaMalloc(&r->master, sizeof(float) * N_PARAMS) == cudaSuccess &&
              cudaMalloc(&r->m1, sizeof(float) * N_PARAMS) == cudaSuccess &&
              cudaMalloc(&r->m2, sizeof(float) * N_PARAMS) == cudaSuccess &&
              cudaMalloc(&r->grads, sizeof(float) * N_PARAMS) == cudaSuccess &&
              cudaMalloc(&r->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&r->w1b, sizeof(__nv_bfloat16) * kH * kInPad) == cudaSuccess &&
              cudaMalloc(&r->w2b, sizeof(__nv_bfloat16) * kH * kH) == cudaSuccess &&
              cudaMalloc(&r->w3b, sizeof(__nv_bfloat16) * kH) == cudaSuccess &&
              cudaMalloc(&r->err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pmh_rerank_destroy(r);
        return pmh_set_error(PMH_ERR_NOMEM, "reranker allocation failed");
    }
    cudaMemset(r->master, 0, sizeof(float) * N_PARAMS);
    cudaMemset(r->m1, 0, sizeof(float) * N_PARAMS);
    cudaMemset(r->m2, 0, sizeof(float) * N_PARAMS);
    cudaMemset(r->err, 0, sizeof(int));
    refresh_bf16_kernel<<<8, 256>>>(r->master, r->w1b, r->w2b, r->w3b);
    g_pmh_launches.fetch_add(1);
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    *out = r;
    return PMH_OK;
}

extern "C" int pmh_rerank_set_weights(pmh_rerank r, const float* h_params)
{
    if (!r || !h_params) return pmh_set_error(PMH_ERR_ARG, "null argument");
    PMH_TRY(pmh_check_device(r->ctx));
    PMH_CUDA_TRY(cudaMemcpy(r->master, h_params, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice));
    PMH_CUDA_TRY(cudaMemset(r->m1, 0, sizeof(float) * N_PARAMS));
    PMH_CUDA_TRY(cudaMemset(r->m2, 0, sizeof(float) * N_PARAMS));
    r->steps = 0;
    refresh_bf16_kernel<<<8, 256>>>(r->master, r->w1b, r->w2b, r->w3b);
    PMH_LAUNCHED("refresh_bf16_kernel");
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    return PMH_OK;
}

extern "C" int pmh_rerank_get_weights(pmh_rerank r, float* h_params)
{
    if (!r || !h_params) return pmh_set_error(PMH_ERR_ARG, "null argument");
    PMH_TRY(pmh_check_device(r->ctx));
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    PMH_CUDA_TRY(cudaMemcpy(h_params, r->master, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost));
    return PMH_OK;
}

extern "C" int pmh_rerank_features(pmh_ctx ctx, pmh_polys queries, pmh_polys db,
                                   const uint32_t* d_qhashes, const uint32_t* d_dbhashes,
                                   const int64_t* d_row_ptr, const int32_t* d_cand, int64_t Q,
                                   const pmh_params* params, uint16_t* d_feat, void* stream)
{
    PMH_TRY(pmh_check_device(ctx));
    PMH_TRY(pmh_check_params(params));
    if (!queries || !db || Q < 0 || Q > queries->n || params->K % 32 != 0 ||
        (Q > 0 && (!d_qhashes || !d_dbhashes || !d_row_ptr || !d_feat)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments (K must be a multiple of 32)");
    if (Q == 0) return PMH_OK;
    return pmh_launch_agree_features(ctx, d_qhashes, d_dbhashes, d_row_ptr, d_cand, Q, INT64_MAX,
                                     params, nullptr, nullptr, d_feat,
                                     FeatSrc{queries->feat, queries->bbox, queries->area2},
                                     FeatSrc{db->feat, db->bbox, db->area2}, nullptr,
                                     (cudaStream_t)stream);
}

// forward pass: the tensor-core kernel (a few CTAs per SM at most, so that their
// tensor-memory allocations, 128 columns each, always fit the SM's 512)
static int tc_forward(pmh_rerank r, const uint16_t* d_feat, int64_t n, float* d_score, int* err,
                      cudaStream_t s)
{
    const size_t smem = std::max<size_t>(sizeof(TcSmem) + 1024, 60 * 1024);
    PMH_CUDA_TRY(cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int blocks = (int)std::min<int64_t>((n + kTcRows - 1) / kTcRows, (int64_t)r->ctx->sm_count);
    mlp_tc_kernel<<<std::max(blocks, 1), kTcThreads, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(d_feat), n, r->w1b, r->w2b, r->w3b, r->master, d_score, err);
    PMH_LAUNCHED("mlp_tc_kernel");
    return PMH_OK;
}

static int train_launch(pmh_rerank r, const uint16_t* d_feat, const float* d_label, int64_t n,
                        cudaStream_t s)
{
    const size_t smem = sizeof(MlpSmem);
    PMH_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int blocks = (int)std::min<int64_t>((n + kChunk - 1) / kChunk, (int64_t)r->ctx->sm_count);
    mlp_train_kernel<<<std::max(blocks, 1), kWarpsMlp * 32, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(d_feat), d_label, n, n, r->w1b, r->w2b, r->w3b,
        r->master, r->grads, r->loss);
    PMH_LAUNCHED("mlp_train_kernel");
    return PMH_OK;
}

int pmh_launch_rerank_forward(pmh_rerank r, const uint16_t* feat, int64_t n_rows, float* score,
                              int* d_flags, cudaStream_t s)
{
    if (n_rows <= 0) return PMH_OK;
    return tc_forward(r, feat, n_rows, score, d_flags, s);
}

bool pmh_rerank_select_fits(int S, int K) { return S >= 4 && S <= kTcRows && kTcRows % S == 0 && K % 32 == 0 && K <= 4096; }

int pmh_launch_rerank_select(pmh_rerank r, const uint32_t* qh, const uint32_t* ph, const int32_t* sl_ids,
                             const int32_t* sl_n, int64_t Q, const int64_t* d_n, int S, int m,
                             const pmh_params* P, FeatSrc qf, FeatSrc pf, int32_t* out_ids, int32_t* out_n,
                             int* d_flags, cudaStream_t s)
{
    if (Q <= 0) return PMH_OK;
    if (!pmh_rerank_select_fits(S, (int)P->K) || m < 1)
        return pmh_set_error(PMH_ERR_ARG, "fused selection: S must divide 128 (S >= 4), K a multiple of 32");
    // at most three CTAs per SM (shared memory), so their tensor-memory allocations
    // (128 columns each) always fit the SM's 512
    const size_t smem = std::max<size_t>(sizeof(SelSmem) + 1024, 60 * 1024);
    auto fn = S % kSelPairs == 0 ? rerank_select_kernel<true> : rerank_select_kernel<false>;
    PMH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the whole carveout as shared memory, so that three CTAs fit an SM
    PMH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 1;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem));
    const int64_t G = kTcRows / S, tiles = (Q + G - 1) / G;
    const int blocks =
        (int)std::min<int64_t>(tiles, (int64_t)std::min(std::max(per_sm, 1), 3) * r->ctx->sm_count);
    fn<<<std::max(blocks, 1), kTcThreads, smem, s>>>(qh, ph, sl_ids, sl_n, Q, d_n, S, m, (int)P->K, P->T, qf, pf,
                                                      r->w1b, r->w2b, r->w3b, r->master, out_ids, out_n, d_flags,
                                                      d_flags);
    PMH_LAUNCHED("rerank_select_kernel");
    return PMH_OK;
}

extern "C" int pmh_rerank_forward(pmh_rerank r, const uint16_t* d_feat, int64_t n_rows,
                                  float* d_score, void* stream)
{
    if (!r || n_rows < 0 || (n_rows > 0 && (!d_feat || !d_score)))
        return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    if (((uintptr_t)d_feat & 15) != 0) return pmh_set_error(PMH_ERR_ARG, "features must be 16-byte aligned");
    PMH_TRY(pmh_check_device(r->ctx));
    if (n_rows == 0) return PMH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PMH_CUDA_TRY(cudaMemsetAsync(r->err, 0, sizeof(int), s));
    PMH_TRY(tc_forward(r, d_feat, n_rows, d_score, r->err, s));
    int h_err = 0;
    PMH_CUDA_TRY(cudaMemcpyAsync(&h_err, r->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PMH_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) return pmh_set_error(PMH_ERR_CUDA, "a tensor-core wait of the forward pass ran out");
    return PMH_OK;
}

extern "C" int pmh_rerank_gradients(pmh_rerank r, const uint16_t* d_feat, const float* d_label,
                                    int64_t n_rows, float* d_grads, float* d_loss, void* stream)
{
    if (!r || n_rows < 1 || !d_feat || !d_label) return pmh_set_error(PMH_ERR_ARG, "bad arguments");
    PMH_TRY(pmh_check_device(r->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    PMH_CUDA_TRY(cudaMemsetAsync(r->grads, 0, sizeof(float) * N_PARAMS, s));
    PMH_CUDA_TRY(cudaMemsetAsync(r->loss, 0, sizeof(float), s));
    PMH_TRY(train_launch(r, d_feat, d_label, n_rows, s));
    if (d_grads)
        PMH_CUDA_TRY(cudaMemcpyAsync(d_grads, r->grads, sizeof(float) * N_PARAMS,
                                     cudaMemcpyDeviceToDevice, s));
    if (d_loss) PMH_CUDA_TRY(cudaMemcpyAsync(d_loss, r->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PMH_OK;
}

extern "C" int pmh_rerank_adam_step(pmh_rerank r, float lr, float beta1, float beta2, float eps,
                                    void* stream)
{
    if (!r) return pmh_set_error(PMH_ERR_ARG, "null reranker");
    PMH_TRY(pmh_check_device(r->ctx));
    cudaStream_t s = (cudaStream_t)stream;
    r->steps += 1;
    float bc1 = 1.f - powf(beta1, (float)r->steps), bc2 = 1.f - powf(beta2, (float)r->steps);
    adam_kernel<<<8, 256, 0, s>>>(r->master, r->m1, r->m2, r->grads, lr, beta1, beta2, eps, bc1, bc2);
    PMH_LAUNCHED("adam_kernel");
    refresh_bf16_kernel<<<8, 256, 0, s>>>(r->master, r->w1b, r->w2b, r->w3b);
    PMH_LAUNCHED("refresh_bf16_kernel");
    return PMH_OK;
}
