// Host side of the tcgen05 BF16 GEMM: tensor-map encoding (driver entry
// point, no libcuda link), tile-width dispatch, and the C-ABI entry point
// st_gemm_bf16.  The learned one-turn spin map builds on gemm_bf16_tn.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "mlp_fused.cuh"
#include "st_internal.cuh"

namespace st {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encoder() {
    if (g_encode) return ST_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        set_error("cuTensorMapEncodeTiled unavailable from the driver");
        return ST_ECUDA;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return ST_OK;
}

// 2D bf16 row-major matrix [rows][cols], box = box_rows x 64 columns,
// 128-byte swizzle.
static int make_tmap(CUtensorMap* tm, const void* base, int rows, int cols, int box_rows) {
    int rc = get_encoder();
    if (rc) return rc;
    if (((uintptr_t)base & 15) || (cols * 2) % 16) {
        set_error("gemm: operand base must be 16-byte aligned and rows a multiple of 16 bytes");
        return ST_EINVAL;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return ST_ECUDA;
    }
    return ST_OK;
}

// Tensor maps depend only on (base, rows, cols, box rows) -- the data is read
// at run time -- so a map stays valid for any buffer at that address with that
// shape.  The network's buffers are fixed: their maps are encoded once.
struct TmapKey {
    const void* base;
    int rows, cols, box_rows;
};
struct TmapEntry {
    TmapKey key;
    CUtensorMap map;
    bool used;
};
static TmapEntry g_tmaps[256];
static std::mutex g_tmap_mu;

static int get_tmap(CUtensorMap* out, const void* base, int rows, int cols, int box_rows) {
    std::lock_guard<std::mutex> lock(g_tmap_mu);
    const size_t h = ((uintptr_t)base >> 8) ^ ((size_t)rows * 131) ^ ((size_t)cols * 7919) ^ (size_t)box_rows;
    for (int probe = 0; probe < 8; ++probe) {
        TmapEntry& e = g_tmaps[(h + probe) & 255];
        if (e.used && e.key.base == base && e.key.rows == rows && e.key.cols == cols && e.key.box_rows == box_rows) {
            *out = e.map;
            return ST_OK;
        }
        if (!e.used) {
            int rc = make_tmap(&e.map, base, rows, cols, box_rows);
            if (rc) return rc;
            e.key = TmapKey{base, rows, cols, box_rows};
            e.used = true;
            *out = e.map;
            return ST_OK;
        }
    }
    // probe window full: encode without caching
    return make_tmap(out, base, rows, cols, box_rows);
}

template <int BN, int ST>
static int launch_gemm_bn(const void* A, const void* B, int M, int N, int K, const GemmEpi& epi, int32_t* status,
                          cudaStream_t stream, int splits) {
    using Cf = GemmCfg<BN, ST>;
    static PerDeviceOnce attr;
    int rc0 = once_per_device(
        attr,
        [] {
            return cudaFuncSetAttribute(gemm_bf16_tn_kernel<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        Cf::SMEM_BYTES);
        },
        "gemm: cudaFuncSetAttribute");
    if (rc0) return rc0;
    CUtensorMap ta, tb;
    int rc = get_tmap(&ta, A, M, K, 128);
    if (rc == ST_OK) rc = get_tmap(&tb, B, N, K, BN);
    if (rc) return rc;
    const int kblocks = K / 64;
    const int per = (kblocks + splits - 1) / splits;
    dim3 grid(M / 128, N / BN, (kblocks + per - 1) / per);
    gemm_bf16_tn_kernel<BN, ST><<<grid, Cf::THREADS, Cf::SMEM_BYTES, stream>>>(ta, tb, K, per, epi, status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "gemm launch");
}

// D = A B^T with the epilogue; M % 128 == 0, K % 64 == 0, N % 16 == 0.
int gemm_bf16_tn(const void* A, const void* B, int M, int N, int K, const GemmEpi& epi, int32_t* status,
                 cudaStream_t stream, int splits) {
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64 || N % 16) {
        set_error("gemm: need M %% 128 == 0, K %% 64 == 0, N %% 16 == 0 (got %d, %d, %d)", M, N, K);
        return ST_EINVAL;
    }
    splits = gemm_split_count(K, splits);
    if (splits > 1 && epi.mode != EPI_F32) {
        set_error("gemm: split-K needs the plain FP32 epilogue");
        return ST_EINVAL;
    }
    // K blocks per CTA decide the pipeline depth.  Short K: 128-wide tiles (3
    // CTAs per SM), or 256-wide tiles (2 CTAs per SM: 97 KB of shared memory and
    // 256 TMEM columns each) when those fit in one wave and the 128-wide ones
    // would need a second, mostly empty one.
    const int kb = K / 64, per = (kb + splits - 1) / splits;
    if (per <= 4) {
        if (N % 256 == 0 && splits == 1) {
            static int sms_cache[kMaxDeviceFlags] = {0};
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDeviceFlags) {
                if (!sms_cache[dev]) cudaDeviceGetAttribute(&sms_cache[dev], cudaDevAttrMultiProcessorCount, dev);
                sms = sms_cache[dev];
            }
            const long tiles256 = (long)(M / 128) * (N / 256);
            if (sms > 0 && tiles256 <= 2L * sms && 2 * tiles256 > 3L * sms)
                return launch_gemm_bn<256, 2>(A, B, M, N, K, epi, status, stream, splits);
        }
        if (N % 128 == 0) return launch_gemm_bn<128, 2>(A, B, M, N, K, epi, status, stream, splits);
        if (N % 64 == 0) return launch_gemm_bn<64, 2>(A, B, M, N, K, epi, status, stream, splits);
        if (N % 32 == 0) return launch_gemm_bn<32, 2>(A, B, M, N, K, epi, status, stream, splits);
        return launch_gemm_bn<16, 2>(A, B, M, N, K, epi, status, stream, splits);
    }
    if (N % 128 == 0) return launch_gemm_bn<128, 4>(A, B, M, N, K, epi, status, stream, splits);
    if (N % 64 == 0) return launch_gemm_bn<64, 4>(A, B, M, N, K, epi, status, stream, splits);
    if (N % 32 == 0) return launch_gemm_bn<32, 4>(A, B, M, N, K, epi, status, stream, splits);
    return launch_gemm_bn<16, 4>(A, B, M, N, K, epi, status, stream, splits);
}

// Fused inference of the five layers (mlp_fused.cuh): X0 [Bp][64] and the
// weights W1 [256][64], W2..W4 [256][256], W5 [16][256] bf16 K-major; bias
// pointers 16-byte aligned (b1..b4); Y [Bp][16] FP32.
int mlp_fused_forward(const void* X0, const void* const W[5], const float* const bias[5], float* Y, int Bp,
                      int32_t* status, cudaStream_t stream) {
    if (Bp <= 0 || Bp % 128) {
        set_error("mlp_fused_forward: rows must be a positive multiple of 128");
        return ST_EINVAL;
    }
    for (int l = 0; l < 4; ++l)
        if ((uintptr_t)bias[l] & 15) {
            set_error("mlp_fused_forward: hidden-layer biases must be 16-byte aligned");
            return ST_EINVAL;
        }
    static PerDeviceOnce attr;
    int rc = once_per_device(
        attr,
        [] {
            return cudaFuncSetAttribute(mlp_fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        MLPF_SMEM_BYTES);
        },
        "mlp_fused_forward: cudaFuncSetAttribute");
    if (rc) return rc;
    CUtensorMap tx, tw[5];
    rc = get_tmap(&tx, X0, Bp, MLP_KIN_FUSED, 128);
    if (rc == ST_OK) rc = get_tmap(&tw[0], W[0], 256, MLP_KIN_FUSED, 256);
    for (int l = 1; l < 4 && rc == ST_OK; ++l) rc = get_tmap(&tw[l], W[l], 256, 256, 256);
    if (rc == ST_OK) rc = get_tmap(&tw[4], W[4], 16, 256, 16);
    if (rc) return rc;
    MlpFusedArgs a;
    for (int l = 0; l < 5; ++l) a.bias[l] = bias[l];
    a.Y = Y;
    a.status = status;
    mlp_fused_forward_kernel<<<Bp / 128, 256, MLPF_SMEM_BYTES, stream>>>(tx, tw[0], tw[1], tw[2], tw[3], tw[4], a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "mlp_fused_forward launch");
}

// out[i] = sum_z ws[z][i] for float4 entries: each block handles 32 consecutive
// entries (one per lane, coalesced 512-byte rows); its 8 warps take the splits
// z = w, w + 8, ... and their partial sums are added in shared memory in a
// fixed order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) split_reduce_kernel(const float4* __restrict__ ws, int splits, int64_t stride4,
                                                           int64_t count4, float4* __restrict__ out) {
    __shared__ float4 part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < count4) {
#pragma unroll 4
        for (int z = w; z < splits; z += 8) {
            const float4 b = ws[(int64_t)z * stride4 + i];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
    }
    part[w][lane] = a;
    __syncthreads();
    if (w == 0 && i < count4) {
        float4 r = part[0][lane];
        for (int k = 1; k < 8; ++k) {
            const float4 b = part[k][lane];
            r.x += b.x;
            r.y += b.y;
            r.z += b.z;
            r.w += b.w;
        }
        out[i] = r;
    }
}

int gemm_split_reduce(const float* ws, int splits, int64_t stride, int64_t count, float* out, cudaStream_t stream) {
    if ((count & 3) || (stride & 3) || ((uintptr_t)ws & 15) || ((uintptr_t)out & 15)) {
        set_error("gemm_split_reduce: counts and pointers must be multiples of 4 floats");
        return ST_EINVAL;
    }
    const int64_t c4 = count / 4;
    split_reduce_kernel<<<(unsigned)((c4 + 31) / 32), 256, 0, stream>>>((const float4*)ws, splits, stride / 4, c4,
                                                                        (float4*)out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "gemm_split_reduce");
}

}  // namespace st

using namespace st;

extern "C" int st_gemm_bf16(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K,
                            const float* bias, int32_t* status, void* cuda_stream) {
    if (!A || !B || !D || !status) {
        set_error("st_gemm_bf16: null pointer");
        return ST_EINVAL;
    }
    if ((uintptr_t)D & 15) {
        set_error("st_gemm_bf16: D must be 16-byte aligned");
        return ST_EINVAL;
    }
    GemmEpi epi;
    memset(&epi, 0, sizeof(epi));
    epi.mode = bias ? EPI_BIAS_F32 : EPI_F32;
    epi.n_valid = N;
    epi.out_f32 = D;
    epi.ld_f32 = N;
    epi.bias = bias;
    return gemm_bf16_tn(A, B, M, N, K, epi, status, (cudaStream_t)cuda_stream);
}

