// Fused inference of the learned spin map's network: all five layers of a
// 128-row tile in one CTA, the activations never leaving the SM.
//
// The activation tile (128 rows x 256 columns, bf16) lives in shared memory
// in the 128-byte-swizzled K-major layout that TMA writes and the tensor core
// reads (four 64-column blocks of 16 KB; in every 1024-byte group of 8 rows
// the 16-byte chunk index is XORed with the row index mod 8).  Per layer:
//   thread 0 loads the layer's weights (bf16, K-major) with TMA -- the next
//   layer's as soon as the tensor core has finished reading this layer's --
//   and issues the tcgen05 MMAs into one 256-column FP32 accumulator in
//   tensor memory; all eight warps then read their TMEM lanes (rows; two warps
//   per lane quarter, each half of the columns), add
//   the bias, apply SiLU, round to bf16 and write the result back into the
//   activation tile in the swizzled layout (a proxy fence makes those stores
//   visible to the tensor core), which is the next layer's A operand.
// The output layer (N = 16, bias only) writes FP32 rows of y.  The arithmetic
// -- bf16 operands, FP32 accumulation in the same K order, the same epilogue
// -- is that of the layer-by-layer GEMMs, so the results are identical.
// Every mbarrier wait is bounded; on expiry the CTA records the status,
// waits once more for work in flight, frees its tensor memory and returns.
// Included by gemm.cu only (the launcher, declared in tc_gemm.cuh, lives
// there with the tensor-map cache).
#pragma once

#include "tc_gemm.cuh"

namespace st {

struct MlpFusedArgs {
    const float* bias[5];   // b1..b4 [256], padded b5 [16]
    float* Y;               // [Bp][16]
    int32_t* status;
};

constexpr int MLP_KIN_FUSED = 64;                    // the first layer's padded input width
constexpr int MLPF_ACT_BYTES = 4 * 128 * 128;        // 4 K blocks of 128 rows x 128 bytes
constexpr int MLPF_WK_BYTES = 256 * 128;             // one K block of a 256-row weight matrix
constexpr int MLPF_SMEM_BYTES = MLPF_ACT_BYTES + 4 * MLPF_WK_BYTES + 1024;   // + alignment slack

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(256, 1)
    mlp_fused_forward_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                             const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmW3,
                             const __grid_constant__ CUtensorMap tmW4, const __grid_constant__ CUtensorMap tmW5,
                             MlpFusedArgs args) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* act = smem;                       // activations, A operand
    unsigned char* wb = smem + MLPF_ACT_BYTES;       // weights, B operand
    __shared__ uint64_t wbar, mbar;
    __shared__ uint32_t tmem_base_s;
    const int warp = threadIdx.x >> 5;
    const int quarter = warp & 3;                    // TMEM lane quarter this warp may read
    const int r = quarter * 32 + (threadIdx.x & 31); // row of the tile = TMEM lane
    const int c_half = (warp >> 2) * 128;            // warps w and w + 4 split the columns
    const int m0 = blockIdx.x * 128;
    const uint64_t limit = 1000000000ull;
    const CUtensorMap* tmW[5] = {&tmW1, &tmW2, &tmW3, &tmW4, &tmW5};

    if (threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        mbar_init(&mbar, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);

    // layer l's weights into wb: K blocks of 64 columns, 256 rows (16 for the output layer)
    auto load_weights = [&](int l) {
        const int kbs = l == 0 ? 1 : 4;
        const int rows = l == 4 ? 16 : 256;
        mbar_arrive_expect_tx(&wbar, (uint32_t)(kbs * rows * 128 + (l == 0 ? 128 * 128 : 0)));
        if (l == 0) tma_load_2d(act, &tmX, 0, m0, &wbar);   // the input tile with the first layer
        for (int kb = 0; kb < kbs; ++kb) tma_load_2d(wb + kb * MLPF_WK_BYTES, tmW[l], kb * 64, 0, &wbar);
    };
    if (threadIdx.x == 0) load_weights(0);

    uint32_t phase = 0;
    bool ok = true;
    for (int l = 0; l < 5 && ok; ++l) {
        const int kbs = l == 0 ? 1 : 4;
        ok = __syncthreads_and(mbar_wait_bounded_parity(&wbar, phase, limit));
        if (!ok) {   // this layer's copies are still in flight: let them land
            mbar_wait_bounded_parity(&wbar, phase, limit);
            break;
        }
        if (threadIdx.x == 0) {
            tc_fence_after();
            for (int kb = 0; kb < kbs; ++kb) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = smem_desc_sw128(act + kb * 128 * 128 + kk * 32);
                    const uint64_t bd = smem_desc_sw128(wb + kb * MLPF_WK_BYTES + kk * 32);
                    const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                    if (l < 4)
                        tc_mma_bf16(tmem, ad, bd, idesc_bf16_f32<128, 256>(), acc);
                    else
                        tc_mma_bf16(tmem, ad, bd, idesc_bf16_f32<128, 16>(), acc);
                }
            }
            tc_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait_bounded_parity(&mbar, phase, limit));
        if (!ok) {   // this layer's MMAs are still in flight: let them finish
            mbar_wait_bounded_parity(&mbar, phase, limit);
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // the tensor core is done with act and wb: fetch the next layer's
        // weights while the epilogue runs
        if (threadIdx.x == 0 && l < 4) load_weights(l + 1);
        const float* bias = args.bias[l];
        if (l < 4) {
#pragma unroll 1
            for (int c0 = c_half; c0 < c_half + 128; c0 += 32) {
                float v[32];
                tmem_load_cols<32>(lane_addr + c0, v);
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 bb = __ldg(reinterpret_cast<const float4*>(bias + c0 + j));
                    v[j] = silu_f(v[j] + bb.x);
                    v[j + 1] = silu_f(v[j + 1] + bb.y);
                    v[j + 2] = silu_f(v[j + 2] + bb.z);
                    v[j + 3] = silu_f(v[j + 3] + bb.w);
                }
                unsigned char* blk = act + (c0 >> 6) * (128 * 128) + r * 128;
                const int chunk0 = (c0 & 63) >> 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 pk;
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * q], v[8 * q + 1]);
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * q + 2], v[8 * q + 3]);
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * q + 4], v[8 * q + 5]);
                    __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * q + 6], v[8 * q + 7]);
                    pk.x = *reinterpret_cast<uint32_t*>(&h0);
                    pk.y = *reinterpret_cast<uint32_t*>(&h1);
                    pk.z = *reinterpret_cast<uint32_t*>(&h2);
                    pk.w = *reinterpret_cast<uint32_t*>(&h3);
                    *reinterpret_cast<uint4*>(blk + (((chunk0 + q) ^ (r & 7)) << 4)) = pk;
                }
            }
            fence_proxy_async_smem();   // the activations are the next MMA's operand
            tc_fence_before();
            __syncthreads();
        } else if (warp < 4) {
            float v[16];
            tmem_load_cols<16>(lane_addr, v);
            float* y = args.Y + (size_t)(m0 + r) * 16;
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(y + j) =
                    make_float4(v[j] + bias[j], v[j + 1] + bias[j + 1], v[j + 2] + bias[j + 2], v[j + 3] + bias[j + 3]);
        }
    }
    if (!ok && threadIdx.x == 0) atomicExch(args.status, STATUS_MMA_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace st
