// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), written
// directly in PTX:  D[M x N] = A[M x K] . B[N x K]^T  (+ fused epilogue),
// A and B bf16 row-major (K contiguous, "K-major" for both operands), FP32
// accumulation in tensor memory (TMEM).
//
// One CTA of 256 threads computes a 128 x BN tile:
//   thread 0   : TMA producer -- 2D tensor-map loads of 64-wide K blocks of A
//                and B into a 2- or 4-stage shared-memory ring, 128-byte swizzle
//                (the canonical K-major SW128 layout the MMA reads directly);
//   thread 32  : MMA issuer -- 4 x tcgen05.mma (K = 16 each) per K block,
//                tcgen05.commit to the stage's "empty" barrier, and to the
//                "done" barrier after the last block;
//   all 8 warps: epilogue -- tcgen05.ld of their 32 TMEM lanes (= rows; warps
//                w and w + 4 share lanes and split the columns),
//                bias / SiLU (and its derivative stored in bf16 for the
//                backward pass) / times the stored SiLU derivative, FP32 or
//                BF16 stores (row-major and, for backward passes, transposed).
// Every mbarrier wait is bounded (about one second); on expiry the CTA sets
// the status word, waits once more for work in flight, frees its TMEM and
// returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace st {

enum GemmEpiMode : int32_t { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_SILU = 2, EPI_DSILU = 3 };

struct GemmEpi {
    int32_t mode;
    int32_t n_valid;                 // columns >= n_valid are written as zero to the bf16 outputs
    float* out_f32;                  // [M][ld_f32]
    int32_t ld_f32;
    const float* bias;               // [N]
    __nv_bfloat16* out_bf16;         // [M][ld_bf16]
    int32_t ld_bf16;
    __nv_bfloat16* out_bf16_t;       // [N][ld_bf16_t] (transposed)
    int32_t ld_bf16_t;
    const __nv_bfloat16* ds_in;      // [M][ld_ds] SiLU derivatives at the pre-activations (EPI_DSILU)
    int32_t ld_ds;
    __nv_bfloat16* ds_out;           // [M][ld_dso] SiLU derivatives, written by EPI_BIAS_SILU
    int32_t ld_dso;
    int64_t split_stride;            // split-K (EPI_F32): split z writes out_f32 + z * split_stride
};

enum { STATUS_MMA_TIMEOUT = 2 };

// D = A B^T with the epilogue (host launcher, gemm.cu); M % 128 == 0,
// K % 64 == 0, N % 16 == 0.  With splits > 1 (EPI_F32 only) the K range is
// cut into that many pieces, piece z written to out_f32 + z * split_stride,
// and the caller reduces them (gemm_split_reduce).
int gemm_bf16_tn(const void* A, const void* B, int M, int N, int K, const GemmEpi& epi, int32_t* status,
                 cudaStream_t stream, int splits = 1);
// Fused inference of the network's five layers (gemm.cu, kernel in
// mlp_fused.cuh): X0 [Bp][64] bf16 input rows, W1 [256][64], W2..W4
// [256][256], W5 [16][256] bf16 K-major, biases b1..b4 [256] (16-byte
// aligned) and b5 [16], Y [Bp][16] FP32; Bp % 128 == 0.
int mlp_fused_forward(const void* X0, const void* const W[5], const float* const bias[5], float* Y, int Bp,
                      int32_t* status, cudaStream_t stream);
// out[i] = sum_z ws[z * stride + i], i < count
int gemm_split_reduce(const float* ws, int splits, int64_t stride, int64_t count, float* out, cudaStream_t stream);
// K blocks per split for a requested split count (every split gets >= 1 block)
inline int gemm_split_count(int K, int want) {
    const int kblocks = K / 64;
    if (want < 1) want = 1;
    if (want > kblocks) want = kblocks;
    const int per = (kblocks + want - 1) / want;
    return (kblocks + per - 1) / per;
}

// ---- tcgen05 / TMA primitives ---------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzled layout: rows of 128 bytes (64 bf16 along K), 8-row atoms of 1024
// bytes (stride byte offset 1024), start address in 16-byte units, version 1,
// layout type 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr & 0x3FFFFull) >> 4;
    d |= 1ull << 16;                       // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset
    d |= 1ull << 46;                       // descriptor version
    d |= 2ull << 61;                       // swizzle mode: 128 B
    return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N.
template <int M, int N>
__host__ __device__ constexpr uint32_t idesc_bf16_f32() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int NC>
__device__ __forceinline__ void tmem_load_cols(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_load_cols<32>(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load_cols<16>(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// SiLU and its derivative.  Their results are rounded to bf16 (8 bits) or
// multiply a gradient that is, so the fast division (2 ulp of FP32) is exact
// enough; for z < -87 the exponential overflows the fast division's range and
// the limits (0) are returned directly.
__device__ __forceinline__ float silu_f(float z) { return z < -87.0f ? 0.0f : __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    if (z < -87.0f) return 0.0f;
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
// SiLU and its derivative from one sigmoid s (a = z s, d = s (1 + z (1 - s)))
__device__ __forceinline__ void silu_dsilu_f(float z, float& a, float& d) {
    const float s = z < -87.0f ? 0.0f : __fdividef(1.0f, 1.0f + __expf(-z));
    a = z * s;
    d = s * (1.0f + z * (1.0f - s));
}

// BN: tile width along N; ST: shared-memory pipeline stages (2 for the short
// K = 64..256 of the network's layers, so that up to 3 CTAs share an SM and
// overlap one tile's epilogue with the next tile's loads and MMAs; 4 for the
// long K ranges of the weight gradients).
template <int BN, int ST>
struct GemmCfg {
    static constexpr int BM = 128, BK = 64, STAGES = ST;
    // 8 warps: warps w and w + 4 read the same 32 TMEM lanes (rows) and split
    // the tile's columns in the epilogue; threads 0 and 32 also run the TMA
    // producer and the MMA issuer before it
    static constexpr int THREADS = 256;
    static constexpr int MIN_BLOCKS = BN >= 256 ? 2 : (ST == 2 ? 3 : 1);
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack
    static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN;        // power of two >= 32
};

template <int BN, int ST>
__global__ void __launch_bounds__(GemmCfg<BN, ST>::THREADS, GemmCfg<BN, ST>::MIN_BLOCKS) gemm_bf16_tn_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, int K,
                                                              int kb_per_split, GemmEpi epi, int32_t* status) {
    using C = GemmCfg<BN, ST>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[C::STAGES], empty_bar[C::STAGES], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int32_t abort_s;
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.x * C::BM;
    const int n0 = blockIdx.y * BN;
    // this CTA's K blocks: [kb0, kb0 + kblocks)
    const int kb0 = blockIdx.z * kb_per_split;
    const int kb_all = K / C::BK;
    const int kblocks = (kb_all - kb0) < kb_per_split ? (kb_all - kb0) : kb_per_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_s = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint64_t limit = 1000000000ull;

    if (threadIdx.x == 0) {
        // TMA producer
        for (int kb = 0; kb < kblocks; ++kb) {
            const int s = kb % C::STAGES;
            if (kb >= C::STAGES) {
                if (!mbar_wait_bounded_parity(&empty_bar[s], ((kb / C::STAGES) - 1) & 1, limit)) {
                    atomicExch(&abort_s, 1);
                    break;
                }
            }
            unsigned char* a = smem + s * C::STAGE_BYTES;
            unsigned char* b = a + C::A_BYTES;
            mbar_arrive_expect_tx(&full_bar[s], C::STAGE_BYTES);
            tma_load_2d(a, &tmA, (kb0 + kb) * C::BK, m0, &full_bar[s]);
            tma_load_2d(b, &tmB, (kb0 + kb) * C::BK, n0, &full_bar[s]);
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_f32<128, BN>();
        for (int kb = 0; kb < kblocks; ++kb) {
            const int s = kb % C::STAGES;
            if (!mbar_wait_bounded_parity(&full_bar[s], (kb / C::STAGES) & 1, limit)) {
                atomicExch(&abort_s, 1);
                break;
            }
            tc_fence_after();
            const unsigned char* a = smem + s * C::STAGE_BYTES;
            const unsigned char* b = a + C::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < C::BK / 16; ++kk)
                tc_mma_bf16(tmem, smem_desc_sw128(a + kk * 32), smem_desc_sw128(b + kk * 32), idesc,
                            (kb > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty_bar[s]);
        }
        tc_commit(&done_bar);
    }
    // epilogue: every thread owns one TMEM lane (= row) of its warp's quarter
    const bool done_ok = mbar_wait_bounded_parity(&done_bar, 0, limit);
    tc_fence_after();
    __syncthreads();
    if (!done_ok || abort_s) {
        if (threadIdx.x == 0) atomicExch(status, STATUS_MMA_TIMEOUT);
        if (!done_ok) mbar_wait_bounded_parity(&done_bar, 0, limit);   // let work in flight drain
    } else {
        const int quarter = warp & 3;                 // TMEM lane quarter this warp may read
        const int row = m0 + quarter * 32 + (threadIdx.x & 31);
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
        // column range of this warp: the first or second half of the tile
        constexpr int NHALF = BN >= 64 ? BN / 2 : BN;
        const int c_begin = BN >= 64 ? (warp >> 2) * NHALF : ((warp >> 2) ? BN : 0);
        const int c_end = BN >= 64 ? c_begin + NHALF : ((warp >> 2) ? BN : BN);
        // the bias is read as 16-byte vectors when it is 16-byte aligned (every
        // column chunk starts at a multiple of 16), element by element otherwise
        const bool bias_v4 = ((uintptr_t)epi.bias & 15) == 0;
        auto bias4 = [&](int c) -> float4 {
            if (bias_v4) return __ldg(reinterpret_cast<const float4*>(epi.bias + c));
            return make_float4(epi.bias[c], epi.bias[c + 1], epi.bias[c + 2], epi.bias[c + 3]);
        };
        constexpr int CH = BN < 32 ? BN : 32;
#pragma unroll 1
        for (int c0 = c_begin; c0 < c_end; c0 += CH) {
            float v[CH];
            tmem_load_cols<CH>(lane_addr + c0, v);
            const int nb = n0 + c0;
            // Row-major outputs are written as 16-byte vectors of the thread's
            // row (CH consecutive columns); the transposed bf16 output is
            // coalesced across the warp's 32 consecutive rows.
            if (epi.mode == EPI_F32 || epi.mode == EPI_BIAS_F32) {
                float* dst = epi.out_f32 + (size_t)blockIdx.z * epi.split_stride + (size_t)row * epi.ld_f32 + nb;
#pragma unroll
                for (int j = 0; j < CH; j += 4) {
                    float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    if (epi.mode == EPI_BIAS_F32) {
                        const float4 bb = bias4(nb + j);
                        o.x += bb.x;
                        o.y += bb.y;
                        o.z += bb.z;
                        o.w += bb.w;
                    }
                    *reinterpret_cast<float4*>(dst + j) = o;
                }
            } else {
                if (epi.mode == EPI_BIAS_SILU) {
#pragma unroll
                    for (int j = 0; j < CH; j += 4) {   // the bias as 16-byte loads (same address across the warp)
                        const float4 bb = bias4(nb + j);
                        v[j] += bb.x;
                        v[j + 1] += bb.y;
                        v[j + 2] += bb.z;
                        v[j + 3] += bb.w;
                    }
                    if (epi.ds_out) {   // SiLU(z), and SiLU'(z) in bf16 for the backward pass
                        __nv_bfloat16* dd = epi.ds_out + (size_t)row * epi.ld_dso + nb;
#pragma unroll
                        for (int j = 0; j < CH; j += 8) {
                            float dv[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) silu_dsilu_f(v[j + k], v[j + k], dv[k]);
                            uint4 pk;
                            __nv_bfloat162 h0 = __floats2bfloat162_rn(dv[0], dv[1]);
                            __nv_bfloat162 h1 = __floats2bfloat162_rn(dv[2], dv[3]);
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(dv[4], dv[5]);
                            __nv_bfloat162 h3 = __floats2bfloat162_rn(dv[6], dv[7]);
                            pk.x = *reinterpret_cast<uint32_t*>(&h0);
                            pk.y = *reinterpret_cast<uint32_t*>(&h1);
                            pk.z = *reinterpret_cast<uint32_t*>(&h2);
                            pk.w = *reinterpret_cast<uint32_t*>(&h3);
                            *reinterpret_cast<uint4*>(dd + j) = pk;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < CH; ++j) v[j] = silu_f(v[j]);
                    }
                } else {   // EPI_DSILU: times the stored SiLU'(z)
                    const __nv_bfloat16* ds = epi.ds_in + (size_t)row * epi.ld_ds + nb;
#pragma unroll
                    for (int j = 0; j < CH; j += 8) {
                        const uint4 q = *reinterpret_cast<const uint4*>(ds + j);
                        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float2 f = __bfloat1622float2(h[k]);
                            v[j + 2 * k] *= f.x;
                            v[j + 2 * k + 1] *= f.y;
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < CH; ++j)
                    if (nb + j >= epi.n_valid) v[j] = 0.0f;
                if (epi.out_bf16) {
                    __nv_bfloat16* bd = epi.out_bf16 + (size_t)row * epi.ld_bf16 + nb;
#pragma unroll
                    for (int j = 0; j < CH; j += 8) {
                        uint4 pk;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[j], v[j + 1]);
                        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[j + 2], v[j + 3]);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[j + 4], v[j + 5]);
                        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[j + 6], v[j + 7]);
                        pk.x = *reinterpret_cast<uint32_t*>(&h0);
                        pk.y = *reinterpret_cast<uint32_t*>(&h1);
                        pk.z = *reinterpret_cast<uint32_t*>(&h2);
                        pk.w = *reinterpret_cast<uint32_t*>(&h3);
                        *reinterpret_cast<uint4*>(bd + j) = pk;
                    }
                }
                if (epi.out_bf16_t) {
                    if constexpr (CH == 32) {
                        // transpose the warp's 32 x 32 block through shared memory (the
                        // pipeline ring is idle once the MMAs are done): lane = row writes
                        // column j of its row at [j][lane], then each lane reads 16 bytes
                        // (8 consecutive rows of one column) and the warp stores 8
                        // transposed rows of 64 bytes per instruction
                        __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(smem) + warp * (32 * 32);
                        const int lane = threadIdx.x & 31;
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 32; ++j) tb[j * 32 + lane] = __float2bfloat16_rn(v[j]);
                        __syncwarp();
                        const int row0 = m0 + quarter * 32;
#pragma unroll
                        for (int it = 0; it < 4; ++it) {
                            const int j = it * 8 + (lane >> 2), seg = lane & 3;
                            const uint4 q = *reinterpret_cast<const uint4*>(tb + j * 32 + seg * 8);
                            *reinterpret_cast<uint4*>(epi.out_bf16_t + (size_t)(nb + j) * epi.ld_bf16_t + row0 + seg * 8) = q;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < CH; ++j)
                            epi.out_bf16_t[(size_t)(nb + j) * epi.ld_bf16_t + row] = __float2bfloat16_rn(v[j]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, C::TMEM_COLS);
}

}  // namespace st
