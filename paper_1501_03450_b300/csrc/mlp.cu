// Host side of the tcgen05 BF16 GEMM: tensor-map encoding (driver entry
// point, no libcuda link), tile-width dispatch, and the C-ABI entry point
// st_gemm_bf16.  The learned one-turn spin map builds on gemm_bf16_tn.
#include <cudaTypedefs.h>

#include <cstring>

#include "st_internal.cuh"
#include "tc_gemm.cuh"

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

template <int BN>
static int launch_gemm_bn(const void* A, const void* B, int M, int N, int K, const GemmEpi& epi, int32_t* status,
                          cudaStream_t stream) {
    using Cf = GemmCfg<BN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tn_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Cf::SMEM_BYTES);
        if (e != cudaSuccess) return cuda_fail(e, "gemm: cudaFuncSetAttribute");
        attr = true;
    }
    CUtensorMap ta, tb;
    int rc = make_tmap(&ta, A, M, K, 128);
    if (rc == ST_OK) rc = make_tmap(&tb, B, N, K, BN);
    if (rc) return rc;
    dim3 grid(M / 128, N / BN);
    gemm_bf16_tn_kernel<BN><<<grid, 128, Cf::SMEM_BYTES, stream>>>(ta, tb, K, epi, status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "gemm launch");
}

// D = A B^T with the epilogue; M % 128 == 0, K % 64 == 0, N % 16 == 0.
int gemm_bf16_tn(const void* A, const void* B, int M, int N, int K, const GemmEpi& epi, int32_t* status,
                 cudaStream_t stream) {
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64 || N % 16) {
        set_error("gemm: need M %% 128 == 0, K %% 64 == 0, N %% 16 == 0 (got %d, %d, %d)", M, N, K);
        return ST_EINVAL;
    }
    if (N % 256 == 0) return launch_gemm_bn<256>(A, B, M, N, K, epi, status, stream);
    if (N % 128 == 0) return launch_gemm_bn<128>(A, B, M, N, K, epi, status, stream);
    if (N % 64 == 0) return launch_gemm_bn<64>(A, B, M, N, K, epi, status, stream);
    if (N % 32 == 0) return launch_gemm_bn<32>(A, B, M, N, K, epi, status, stream);
    return launch_gemm_bn<16>(A, B, M, N, K, epi, status, stream);
}

}  // namespace st

using namespace st;

extern "C" int st_gemm_bf16(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K,
                            const float* bias, int32_t* status, void* cuda_stream) {
    if (!A || !B || !D || !status) {
        set_error("st_gemm_bf16: null pointer");
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

// ===========================================================================
// Learned one-turn spin map: MLP 6 -> 256 -> 256 -> 256 -> 256 -> 4 with SiLU,
// bf16 weights and activations on the tensor cores (gemm_bf16_tn), FP32
// accumulation, FP32 master weights and Adam moments.  Head: the network's
// 4 outputs y give the one-turn quaternion
//     q = normalise(q0 + L x + s y),
// q0 the closed-orbit one-turn quaternion, L x a linear term fitted in FP64
// (optional), s an output scale, x the input scaled per coordinate.
// ===========================================================================
namespace st {

constexpr int MLP_IN = 6, MLP_H = 256, MLP_OUT = 4, MLP_KIN = 64, MLP_NOUT = 16;

// flattened FP32 parameter layout: W1 [256][6], b1, W2 [256][256], b2, W3, b3,
// W4, b4, W5 [4][256], b5
__host__ __device__ constexpr int64_t mlp_w_off(int l) {
    return l == 0 ? 0 : l == 1 ? 1792 : l == 2 ? 67584 : l == 3 ? 133376 : 199168;
}
__host__ __device__ constexpr int64_t mlp_b_off(int l) {
    return l == 0 ? 1536 : l == 1 ? 67328 : l == 2 ? 133120 : l == 3 ? 198912 : 200192;
}
constexpr int64_t MLP_PARAMS = 200196;
static_assert(mlp_b_off(0) == MLP_H * MLP_IN && mlp_w_off(1) == mlp_b_off(0) + MLP_H &&
                  mlp_b_off(1) == mlp_w_off(1) + MLP_H * MLP_H && mlp_w_off(2) == mlp_b_off(1) + MLP_H &&
                  mlp_b_off(2) == mlp_w_off(2) + MLP_H * MLP_H && mlp_w_off(3) == mlp_b_off(2) + MLP_H &&
                  mlp_b_off(3) == mlp_w_off(3) + MLP_H * MLP_H && mlp_w_off(4) == mlp_b_off(3) + MLP_H &&
                  mlp_b_off(4) == mlp_w_off(4) + MLP_OUT * MLP_H && MLP_PARAMS == mlp_b_off(4) + MLP_OUT,
              "parameter layout");

struct MlpHead {
    float q0[4];
    float lin[4][6];
    float scale;
    float in_scale[6];
};

// the head's reference quaternion and input scales in FP64 (linear fit)
struct MlpHeadD {
    double q0[4];
    double in_scale[6];
};

}  // namespace st

struct st_mlp {
    int32_t max_batch = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __nv_bfloat16 *W1p = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr, *W5p = nullptr;
    __nv_bfloat16 *W2T = nullptr, *W3T = nullptr, *W4T = nullptr, *W5Tp = nullptr;
    float* Xf = nullptr;                                    // [B][6] scaled inputs (fp32)
    __nv_bfloat16 *X0 = nullptr, *X0T = nullptr;
    __nv_bfloat16* A[4] = {nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16* AT[4] = {nullptr, nullptr, nullptr, nullptr};
    float* Z[4] = {nullptr, nullptr, nullptr, nullptr};
    float* Y = nullptr;                                     // [B][16]
    __nv_bfloat16 *dYp = nullptr, *dYT = nullptr;
    __nv_bfloat16* dZ[2] = {nullptr, nullptr};
    __nv_bfloat16* dZT[2] = {nullptr, nullptr};
    float* dWtmp = nullptr;                                 // [256][64]
    float* b5p = nullptr;                                   // [16] output bias, zero padded
    double* loss = nullptr;
    int32_t* status = nullptr;
    st::MlpHead head;
    st::MlpHeadD head_d;
    int64_t step = 0;
    bool have_grads = false;
};

namespace st {

__global__ void mlp_pack_x(const float* __restrict__ x, int B, int Bp, MlpHead hd, float* __restrict__ Xf,
                           __nv_bfloat16* __restrict__ X0, __nv_bfloat16* __restrict__ X0T) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bp) return;
    for (int c = 0; c < MLP_KIN; ++c) {
        float v = 0.0f;
        if (r < B && c < MLP_IN) v = x[(size_t)r * MLP_IN + c] * hd.in_scale[c];
        if (c < MLP_IN) Xf[(size_t)r * MLP_IN + c] = v;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        X0[(size_t)r * MLP_KIN + c] = b;
        X0T[(size_t)c * Bp + r] = b;
    }
}

// the same from the tracker's FP64 pair-SoA state (coordinates X..Pt)
__global__ void mlp_pack_state(const double2* __restrict__ xpx, const double2* __restrict__ ypy,
                               const double2* __restrict__ tpt, int B, int Bp, MlpHead hd, float* __restrict__ Xf,
                               __nv_bfloat16* __restrict__ X0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bp) return;
    float z[6] = {0, 0, 0, 0, 0, 0};
    if (r < B) {
        const double2 a = xpx[r], b = ypy[r], c = tpt[r];
        z[0] = (float)a.x;
        z[1] = (float)a.y;
        z[2] = (float)b.x;
        z[3] = (float)b.y;
        z[4] = (float)c.x;
        z[5] = (float)c.y;
    }
    for (int c = 0; c < MLP_KIN; ++c) {
        const float v = c < MLP_IN ? z[c] * hd.in_scale[c] : 0.0f;
        if (c < MLP_IN) Xf[(size_t)r * MLP_IN + c] = v;
        X0[(size_t)r * MLP_KIN + c] = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ void head_quat(const MlpHead& hd, const float* xs, const float* y, float* u) {
    for (int k = 0; k < 4; ++k) {
        float a = hd.q0[k] + hd.scale * y[k];
        for (int c = 0; c < MLP_IN; ++c) a = fmaf(hd.lin[k][c], xs[c], a);
        u[k] = a;
    }
}

// normalised quaternions; with targets also the loss (sum over rows) and
// dL/dy into dYp [Bp][64] and dYT [16][Bp] (bf16, zero padded)
__global__ void mlp_head(const float* __restrict__ Y, const float* __restrict__ Xf, int B, int Bp, MlpHead hd,
                         const float* __restrict__ qt, float* __restrict__ q_out, double* __restrict__ loss,
                         __nv_bfloat16* __restrict__ dYp, __nv_bfloat16* __restrict__ dYT) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (r < Bp) {
        float gy[4] = {0, 0, 0, 0};
        if (r < B) {
            float y[4], xs[6], u[4];
            for (int k = 0; k < 4; ++k) y[k] = Y[(size_t)r * MLP_NOUT + k];
            for (int c = 0; c < MLP_IN; ++c) xs[c] = Xf[(size_t)r * MLP_IN + c];
            head_quat(hd, xs, y, u);
            const float n = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
            const float in = 1.0f / n;
            float q[4];
            for (int k = 0; k < 4; ++k) q[k] = u[k] * in;
            if (q_out)
                for (int k = 0; k < 4; ++k) q_out[(size_t)r * 4 + k] = q[k];
            if (qt) {
                float d[4], dq = 0.0f;
                for (int k = 0; k < 4; ++k) {
                    d[k] = q[k] - qt[(size_t)r * 4 + k];
                    l += d[k] * d[k];
                }
                // dL/dq = 2 d / B; dL/du = (I - q q^T) dL/dq / |u|; dL/dy = s dL/du
                for (int k = 0; k < 4; ++k) dq += q[k] * d[k];
                for (int k = 0; k < 4; ++k) gy[k] = hd.scale * (2.0f / B) * (d[k] - q[k] * dq) * in;
            }
        }
        if (dYp)
            for (int c = 0; c < MLP_KIN; ++c)
                dYp[(size_t)r * MLP_KIN + c] = __float2bfloat16_rn(c < 4 ? gy[c] : 0.0f);
        if (dYT)
            for (int c = 0; c < MLP_NOUT; ++c) dYT[(size_t)c * Bp + r] = __float2bfloat16_rn(c < 4 ? gy[c] : 0.0f);
    }
    if (loss) {
        // block reduction, one double atomic per block
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        __shared__ float part[32];
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            atomicAdd(loss, (double)t / B);
        }
    }
}

// row sums of a [rows][Bp] bf16 matrix (bias gradients), one warp per row
__global__ void mlp_rowsum(const __nv_bfloat16* __restrict__ M, int rows, int Bp, float* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    float s = 0.0f;
    for (int c = threadIdx.x & 31; c < Bp; c += 32) s += __bfloat162float(M[(size_t)row * Bp + c]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) out[row] = s;
}

// dW1 [256][6] from dWtmp [256][64]; dW5 [4][256] from D' [256][16] (transposed)
__global__ void mlp_gather_w1(const float* __restrict__ tmp, float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_H * MLP_IN) return;
    g[i] = tmp[(i / MLP_IN) * MLP_KIN + (i % MLP_IN)];
}
__global__ void mlp_gather_w5(const float* __restrict__ tmp, float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_OUT * MLP_H) return;
    const int o = i / MLP_H, in = i % MLP_H;
    g[i] = tmp[in * MLP_NOUT + o];
}

// Refresh the bf16 weight copies (padded, and transposed for the backward
// pass) from the FP32 master parameters.
__global__ void mlp_cast_weights(const float* __restrict__ p, __nv_bfloat16* W1p, __nv_bfloat16* W2,
                                 __nv_bfloat16* W3, __nv_bfloat16* W4, __nv_bfloat16* W5p, __nv_bfloat16* W2T,
                                 __nv_bfloat16* W3T, __nv_bfloat16* W4T, __nv_bfloat16* W5Tp, float* b5p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NOUT) b5p[i] = i < MLP_OUT ? p[mlp_b_off(4) + i] : 0.0f;
    // W1p [256][64]
    if (i < MLP_H * MLP_KIN) {
        const int r = i / MLP_KIN, c = i % MLP_KIN;
        W1p[i] = __float2bfloat16_rn(c < MLP_IN ? p[mlp_w_off(0) + r * MLP_IN + c] : 0.0f);
    }
    if (i < MLP_H * MLP_H) {
        const int r = i / MLP_H, c = i % MLP_H;
        __nv_bfloat16* Ws[3] = {W2, W3, W4};
        __nv_bfloat16* WTs[3] = {W2T, W3T, W4T};
        for (int l = 0; l < 3; ++l) {
            const __nv_bfloat16 b = __float2bfloat16_rn(p[mlp_w_off(l + 1) + i]);
            Ws[l][i] = b;
            WTs[l][(size_t)c * MLP_H + r] = b;
        }
    }
    // W5p [16][256]
    if (i < MLP_NOUT * MLP_H) {
        const int r = i / MLP_H, c = i % MLP_H;
        W5p[i] = __float2bfloat16_rn(r < MLP_OUT ? p[mlp_w_off(4) + r * MLP_H + c] : 0.0f);
    }
    // W5Tp [256][64]
    if (i < MLP_H * MLP_KIN) {
        const int r = i / MLP_KIN, c = i % MLP_KIN;
        W5Tp[i] = __float2bfloat16_rn(c < MLP_OUT ? p[mlp_w_off(4) + c * MLP_H + r] : 0.0f);
    }
}

__global__ void mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                         const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                         float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Spin step of the learned map: q = normalise(q0 + L x + s y) (in FP64 from
// the FP32 network output), S <- q S conj(q); optional running sum of S.
__global__ void surrogate_apply(const float* __restrict__ Y, const float* __restrict__ Xf, int B, MlpHead hd,
                                double2* __restrict__ sxy, double* __restrict__ szp, const uint8_t* __restrict__ lost,
                                double* __restrict__ sum) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B || lost[r]) return;
    float y[4], xs[6], u[4];
    for (int k = 0; k < 4; ++k) y[k] = Y[(size_t)r * MLP_NOUT + k];
    for (int c = 0; c < MLP_IN; ++c) xs[c] = Xf[(size_t)r * MLP_IN + c];
    head_quat(hd, xs, y, u);
    Quat q{(double)u[0], (double)u[1], (double)u[2], (double)u[3]};
    q = qnormalize(q);
    double2 a = sxy[r];
    double sx = a.x, sy = a.y, sz = szp[r];
    rotate_vec(q, sx, sy, sz);
    sxy[r] = make_double2(sx, sy);
    szp[r] = sz;
    if (sum) {
        sum[r] += sx;
        sum[(size_t)B + r] += sy;
        sum[2 * (size_t)B + r] += sz;
    }
}

// Training pairs from the tracker's SoA FP64 buffers (z [6][n] before the
// turn, q [4][n] its one-turn quaternion) into the network's FP32 rows.
__global__ void mlp_pack_pairs(const double* __restrict__ z, const double* __restrict__ q, int64_t n,
                               float* __restrict__ x_rows, float* __restrict__ q_rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < MLP_IN; ++c) x_rows[i * MLP_IN + c] = (float)z[c * n + i];
    for (int k = 0; k < 4; ++k) q_rows[i * 4 + k] = (float)q[k * n + i];
}

// FP64 moments of the least-squares fit q - q0 ~ c + L xs over the tracked
// pairs: features f = (1, xs), G = sum f f^T (7x7), H = sum f (q - q0)^T (7x4),
// packed as 49 + 28 doubles; one atomic add per value and block.
constexpr int FIT_F = 1 + MLP_IN, FIT_M = FIT_F * FIT_F + FIT_F * 4;

__global__ void __launch_bounds__(256) mlp_fit_moments(const double* __restrict__ z, const double* __restrict__ q,
                                                       const uint8_t* __restrict__ lost, int64_t n, MlpHeadD hd,
                                                       double* __restrict__ mom) {
    double G[FIT_F][FIT_F], H[FIT_F][4];
#pragma unroll
    for (int a = 0; a < FIT_F; ++a) {
        for (int b = 0; b < FIT_F; ++b) G[a][b] = 0.0;
        for (int k = 0; k < 4; ++k) H[a][k] = 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (lost && lost[i]) continue;
        double f[FIT_F];
        f[0] = 1.0;
        for (int c = 0; c < MLP_IN; ++c) f[1 + c] = z[c * n + i] * hd.in_scale[c];
        double r[4];
        for (int k = 0; k < 4; ++k) r[k] = q[k * n + i] - hd.q0[k];
#pragma unroll
        for (int a = 0; a < FIT_F; ++a) {
#pragma unroll
            for (int b = a; b < FIT_F; ++b) G[a][b] = fma(f[a], f[b], G[a][b]);
#pragma unroll
            for (int k = 0; k < 4; ++k) H[a][k] = fma(f[a], r[k], H[a][k]);
        }
    }
    __shared__ double red[8];
    auto block_sum = [&](double v, double* dst) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            atomicAdd(dst, t);
        }
    };
#pragma unroll
    for (int a = 0; a < FIT_F; ++a)
#pragma unroll
        for (int b = a; b < FIT_F; ++b) block_sum(G[a][b], &mom[a * FIT_F + b]);
#pragma unroll
    for (int a = 0; a < FIT_F; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) block_sum(H[a][k], &mom[FIT_F * FIT_F + a * 4 + k]);
}

static GemmEpi epi_base() {
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    return e;
}

static int mlp_refresh_weights(st_mlp* n) {
    const int total = MLP_H * MLP_H;
    mlp_cast_weights<<<(total + 255) / 256, 256, 0, n->stream>>>(n->p, n->W1p, n->W2, n->W3, n->W4, n->W5p, n->W2T,
                                                                 n->W3T, n->W4T, n->W5Tp, n->b5p);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "mlp: weight cast");
}

// forward through the five layers from X0 (rows Bp); keep_t writes the
// transposed activations for a following backward pass
static int mlp_forward_layers(st_mlp* n, int Bp, bool keep_t) {
    int rc;
    GemmEpi e = epi_base();
    const __nv_bfloat16* Win[4] = {n->W1p, n->W2, n->W3, n->W4};
    const __nv_bfloat16* in = n->X0;
    int K = MLP_KIN;
    for (int l = 0; l < 4; ++l) {
        e = epi_base();
        e.mode = EPI_BIAS_SILU;
        e.n_valid = MLP_H;
        e.bias = n->p + mlp_b_off(l);
        e.out_bf16 = n->A[l];
        e.ld_bf16 = MLP_H;
        e.out_bf16_t = keep_t ? n->AT[l] : nullptr;
        e.ld_bf16_t = Bp;
        e.z_out = keep_t ? n->Z[l] : nullptr;
        e.ld_zo = MLP_H;
        rc = gemm_bf16_tn(in, Win[l], Bp, MLP_H, K, e, n->status, n->stream);
        if (rc) return rc;
        in = n->A[l];
        K = MLP_H;
    }
    e = epi_base();
    e.mode = EPI_BIAS_F32;
    e.n_valid = MLP_NOUT;
    e.out_f32 = n->Y;
    e.ld_f32 = MLP_NOUT;
    // bias of the padded output layer: b5 for the first 4 columns, 0 after
    e.bias = n->b5p;
    return gemm_bf16_tn(in, n->W5p, Bp, MLP_NOUT, MLP_H, e, n->status, n->stream);
}

static int check_status(st_mlp* n, const char* what) {
    int32_t st_h = 0;
    cudaError_t e = cudaMemcpyAsync(&st_h, n->status, sizeof(int32_t), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (st_h) {
        set_error("%s: a tensor-core kernel reported status %d (bounded wait expired)", what, st_h);
        return ST_ETIMEOUT;
    }
    return ST_OK;
}

}  // namespace st

extern "C" {

int64_t st_mlp_param_count(void) { return st::MLP_PARAMS; }

int st_mlp_destroy(st_mlp* n) {
    if (!n) return ST_OK;
    cudaStreamSynchronize(n->stream);
    void* ptrs[] = {n->p, n->m, n->v, n->g, n->W1p, n->W2, n->W3, n->W4, n->W5p, n->W2T, n->W3T, n->W4T, n->W5Tp,
                    n->Xf, n->X0, n->X0T, n->Y, n->dYp, n->dYT, n->dWtmp, n->b5p, n->loss, n->status};
    for (void* q : ptrs) cudaFree(q);
    for (int l = 0; l < 4; ++l) {
        cudaFree(n->A[l]);
        cudaFree(n->AT[l]);
        cudaFree(n->Z[l]);
    }
    for (int k = 0; k < 2; ++k) {
        cudaFree(n->dZ[k]);
        cudaFree(n->dZT[k]);
    }
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
    return ST_OK;
}

int st_mlp_create(int32_t max_batch, void* cuda_stream, st_mlp** out) {
    if (!out || max_batch < 1 || max_batch > (1 << 22)) {
        set_error("st_mlp_create: need 1 <= max_batch <= 2^22");
        return ST_EINVAL;
    }
    st_mlp* n = new (std::nothrow) st_mlp();
    if (!n) {
        set_error("st_mlp_create: host allocation failed");
        return ST_ENOMEM;
    }
    const int Bp = ((max_batch + 127) / 128) * 128;
    n->max_batch = Bp;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        n->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete n;
            return cuda_fail(e, "st_mlp_create: stream");
        }
        n->own_stream = true;
    }
    const size_t P = (size_t)MLP_PARAMS;
    const size_t bf = sizeof(__nv_bfloat16);
#define ST_MALLOC(ptr, bytes)                                                                                   \
    e = cudaMalloc((void**)&(ptr), (bytes));                                                                    \
    if (e != cudaSuccess) {                                                                                     \
        st_mlp_destroy(n);                                                                                      \
        set_error("st_mlp_create: cudaMalloc of %zu bytes failed: %s", (size_t)(bytes), cudaGetErrorString(e)); \
        return ST_ENOMEM;                                                                                       \
    }
    ST_MALLOC(n->p, P * 4);
    ST_MALLOC(n->m, P * 4);
    ST_MALLOC(n->v, P * 4);
    ST_MALLOC(n->g, P * 4);
    ST_MALLOC(n->W1p, (size_t)MLP_H * MLP_KIN * bf);
    ST_MALLOC(n->W2, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W3, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W4, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W5p, (size_t)MLP_NOUT * MLP_H * bf);
    ST_MALLOC(n->W2T, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W3T, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W4T, (size_t)MLP_H * MLP_H * bf);
    ST_MALLOC(n->W5Tp, (size_t)MLP_H * MLP_KIN * bf);
    ST_MALLOC(n->Xf, (size_t)Bp * MLP_IN * 4);
    ST_MALLOC(n->X0, (size_t)Bp * MLP_KIN * bf);
    ST_MALLOC(n->X0T, (size_t)Bp * MLP_KIN * bf);
    for (int l = 0; l < 4; ++l) {
        ST_MALLOC(n->A[l], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->AT[l], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->Z[l], (size_t)Bp * MLP_H * 4);
    }
    ST_MALLOC(n->Y, (size_t)Bp * MLP_NOUT * 4);
    ST_MALLOC(n->dYp, (size_t)Bp * MLP_KIN * bf);
    ST_MALLOC(n->dYT, (size_t)Bp * MLP_NOUT * bf);
    for (int k = 0; k < 2; ++k) {
        ST_MALLOC(n->dZ[k], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->dZT[k], (size_t)Bp * MLP_H * bf);
    }
    ST_MALLOC(n->dWtmp, (size_t)MLP_H * MLP_KIN * 4);
    ST_MALLOC(n->b5p, MLP_NOUT * 4);
    ST_MALLOC(n->loss, sizeof(double));
    ST_MALLOC(n->status, sizeof(int32_t));
#undef ST_MALLOC
    e = cudaMemset(n->p, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(n->g, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(n->status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        st_mlp_destroy(n);
        return cuda_fail(e, "st_mlp_create: init");
    }
    memset(&n->head, 0, sizeof(n->head));
    n->head.q0[0] = 1.0f;
    n->head.scale = 1.0f;
    for (int c = 0; c < MLP_IN; ++c) n->head.in_scale[c] = 1.0f;
    int rc = mlp_refresh_weights(n);
    if (rc) {
        st_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return ST_OK;
}

int st_mlp_set_params(st_mlp* n, const float* params) {
    if (!n || !params) {
        set_error("st_mlp_set_params: null pointer");
        return ST_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(n->p, params, (size_t)MLP_PARAMS * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, (size_t)MLP_PARAMS * 4, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, (size_t)MLP_PARAMS * 4, n->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_set_params");
    n->step = 0;
    int rc = mlp_refresh_weights(n);
    if (rc) return rc;
    e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_set_params: sync");
}

int st_mlp_get_params(st_mlp* n, float* params) {
    if (!n || !params) {
        set_error("st_mlp_get_params: null pointer");
        return ST_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(params, n->p, (size_t)MLP_PARAMS * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_get_params");
}

int st_mlp_set_head(st_mlp* n, const double* q0, const double* lin, double out_scale, const double* in_scale) {
    if (!n || !q0 || !in_scale || !(out_scale > 0.0)) {
        set_error("st_mlp_set_head: null pointer or out_scale <= 0");
        return ST_EINVAL;
    }
    for (int k = 0; k < 4; ++k) {
        n->head.q0[k] = (float)q0[k];
        for (int c = 0; c < MLP_IN; ++c) n->head.lin[k][c] = lin ? (float)lin[k * MLP_IN + c] : 0.0f;
    }
    n->head.scale = (float)out_scale;
    for (int c = 0; c < MLP_IN; ++c) n->head.in_scale[c] = (float)in_scale[c];
    for (int k = 0; k < 4; ++k) n->head_d.q0[k] = q0[k];
    for (int c = 0; c < MLP_IN; ++c) n->head_d.in_scale[c] = in_scale[c];
    return ST_OK;
}

int st_mlp_pack_pairs(const double* z_soa, const double* q_soa, int64_t n, float* x_rows, float* q_rows,
                      void* cuda_stream) {
    if (!z_soa || !q_soa || !x_rows || !q_rows || n < 1) {
        set_error("st_mlp_pack_pairs: null pointer or n < 1");
        return ST_EINVAL;
    }
    mlp_pack_pairs<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(z_soa, q_soa, n, x_rows,
                                                                                       q_rows);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_pack_pairs");
}

int st_mlp_fit_linear(st_mlp* nw, const double* z_soa, const double* q_soa, const uint8_t* lost, int64_t n,
                      double* lin_out) {
    if (!nw || !z_soa || !q_soa || !lin_out || n < 1) {
        set_error("st_mlp_fit_linear: null pointer or n < 1");
        return ST_EINVAL;
    }
    double* d_mom = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_mom, FIT_M * sizeof(double), nw->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_fit_linear: allocation");
    double mom[FIT_M];
    e = cudaMemsetAsync(d_mom, 0, FIT_M * sizeof(double), nw->stream);
    if (e == cudaSuccess) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (n + 255) / 256;
        if (blocks > 4 * sms) blocks = 4 * sms;
        mlp_fit_moments<<<(unsigned)blocks, 256, 0, nw->stream>>>(z_soa, q_soa, lost, n, nw->head_d, d_mom);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mom, d_mom, sizeof(mom), cudaMemcpyDeviceToHost, nw->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nw->stream);
    cudaFreeAsync(d_mom, nw->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_fit_linear");
    // Normal equations over the features with nonzero variance (an input
    // scale of 0 removes its coordinate), solved by Cholesky in FP64.
    double G[FIT_F][FIT_F];
    for (int a = 0; a < FIT_F; ++a)
        for (int b = a; b < FIT_F; ++b) G[a][b] = G[b][a] = mom[a * FIT_F + b];
    int idx[FIT_F], m = 0;
    for (int a = 0; a < FIT_F; ++a)
        if (G[a][a] > 0.0) idx[m++] = a;
    double C[FIT_F][FIT_F] = {};
    for (int a = 0; a < m; ++a) {
        for (int b = 0; b <= a; ++b) {
            double t = G[idx[a]][idx[b]];
            for (int c = 0; c < b; ++c) t -= C[a][c] * C[b][c];
            if (a == b) {
                if (!(t > 0.0)) {
                    set_error("st_mlp_fit_linear: singular normal equations");
                    return ST_EINVAL;
                }
                C[a][a] = sqrt(t);
            } else {
                C[a][b] = t / C[b][b];
            }
        }
    }
    for (int k = 0; k < 4 * MLP_IN; ++k) lin_out[k] = 0.0;
    for (int k = 0; k < 4; ++k) {
        double y[FIT_F], sol[FIT_F];
        for (int a = 0; a < m; ++a) {
            double t = mom[FIT_F * FIT_F + idx[a] * 4 + k];
            for (int c = 0; c < a; ++c) t -= C[a][c] * y[c];
            y[a] = t / C[a][a];
        }
        for (int a = m - 1; a >= 0; --a) {
            double t = y[a];
            for (int c = a + 1; c < m; ++c) t -= C[c][a] * sol[c];
            sol[a] = t / C[a][a];
        }
        for (int a = 0; a < m; ++a)
            if (idx[a] > 0) lin_out[k * MLP_IN + idx[a] - 1] = sol[a];
    }
    return ST_OK;
}

int st_mlp_forward(st_mlp* n, const float* x, int32_t B, float* q_out) {
    if (!n || !x || !q_out || B < 1 || B > n->max_batch) {
        set_error("st_mlp_forward: null pointer or batch outside 1..max_batch");
        return ST_EINVAL;
    }
    const int Bp = ((B + 127) / 128) * 128;
    mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x, B, Bp, n->head, n->Xf, n->X0, n->X0T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_forward: pack");
    int rc = mlp_forward_layers(n, Bp, false);
    if (rc) return rc;
    mlp_head<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, n->Xf, B, Bp, n->head, nullptr, q_out, nullptr, nullptr,
                                                      nullptr);
    e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_forward: head");
}

int st_mlp_loss_grad(st_mlp* n, const float* x, const float* q_target, int32_t B, float* loss, float* grads) {
    if (!n || !x || !q_target || B < 1 || B > n->max_batch) {
        set_error("st_mlp_loss_grad: null pointer or batch outside 1..max_batch");
        return ST_EINVAL;
    }
    const int Bp = ((B + 127) / 128) * 128;
    cudaError_t e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: reset");
    mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x, B, Bp, n->head, n->Xf, n->X0, n->X0T);
    int rc = mlp_forward_layers(n, Bp, true);
    if (rc) return rc;
    mlp_head<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, n->Xf, B, Bp, n->head, q_target, nullptr, n->loss, n->dYp,
                                                      n->dYT);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: head");
    float* g = n->g;
    // layer 5: dW5^T = A4^T . dY  (D'[256][16]), db5 = sum dY, dZ4 = (dY W5) * silu'(Z4)
    GemmEpi ep = epi_base();
    ep.mode = EPI_F32;
    ep.n_valid = MLP_NOUT;
    ep.out_f32 = n->dWtmp;
    ep.ld_f32 = MLP_NOUT;
    rc = gemm_bf16_tn(n->AT[3], n->dYT, MLP_H, MLP_NOUT, Bp, ep, n->status, n->stream);
    if (rc) return rc;
    mlp_gather_w5<<<(MLP_OUT * MLP_H + 255) / 256, 256, 0, n->stream>>>(n->dWtmp, g + mlp_w_off(4));
    mlp_rowsum<<<1, 128, 0, n->stream>>>(n->dYT, MLP_OUT, Bp, g + mlp_b_off(4));
    ep = epi_base();
    ep.mode = EPI_DSILU;
    ep.n_valid = MLP_H;
    ep.z_in = n->Z[3];
    ep.ld_z = MLP_H;
    ep.out_bf16 = n->dZ[0];
    ep.ld_bf16 = MLP_H;
    ep.out_bf16_t = n->dZT[0];
    ep.ld_bf16_t = Bp;
    rc = gemm_bf16_tn(n->dYp, n->W5Tp, Bp, MLP_H, MLP_KIN, ep, n->status, n->stream);
    if (rc) return rc;
    // hidden layers l = 3, 2, 1 (0-based weights W[l], activations A[l-1])
    const __nv_bfloat16* WT[4] = {nullptr, n->W2T, n->W3T, n->W4T};
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        // dW_l = dZ_l^T . A_{l-1}  ->  [256 out][256 in], straight into the gradient buffer
        ep = epi_base();
        ep.mode = EPI_F32;
        ep.n_valid = MLP_H;
        ep.out_f32 = g + mlp_w_off(l);
        ep.ld_f32 = MLP_H;
        rc = gemm_bf16_tn(n->dZT[cur], n->AT[l - 1], MLP_H, MLP_H, Bp, ep, n->status, n->stream);
        if (rc) return rc;
        mlp_rowsum<<<MLP_H / 4, 128, 0, n->stream>>>(n->dZT[cur], MLP_H, Bp, g + mlp_b_off(l));
        // dZ_{l-1} = (dZ_l W_l) * silu'(Z_{l-1})
        ep = epi_base();
        ep.mode = EPI_DSILU;
        ep.n_valid = MLP_H;
        ep.z_in = n->Z[l - 1];
        ep.ld_z = MLP_H;
        ep.out_bf16 = n->dZ[1 - cur];
        ep.ld_bf16 = MLP_H;
        ep.out_bf16_t = n->dZT[1 - cur];
        ep.ld_bf16_t = Bp;
        rc = gemm_bf16_tn(n->dZ[cur], WT[l], Bp, MLP_H, MLP_H, ep, n->status, n->stream);
        if (rc) return rc;
        cur = 1 - cur;
    }
    // layer 1: dW1 = dZ1^T . X0 -> [256][64] -> [256][6]; db1
    ep = epi_base();
    ep.mode = EPI_F32;
    ep.n_valid = MLP_KIN;
    ep.out_f32 = n->dWtmp;
    ep.ld_f32 = MLP_KIN;
    rc = gemm_bf16_tn(n->dZT[cur], n->X0T, MLP_H, MLP_KIN, Bp, ep, n->status, n->stream);
    if (rc) return rc;
    mlp_gather_w1<<<(MLP_H * MLP_IN + 255) / 256, 256, 0, n->stream>>>(n->dWtmp, g + mlp_w_off(0));
    mlp_rowsum<<<MLP_H / 4, 128, 0, n->stream>>>(n->dZT[cur], MLP_H, Bp, g + mlp_b_off(0));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: backward");
    n->have_grads = true;
    if (loss || grads) {
        double lh = 0.0;
        if (loss) e = cudaMemcpyAsync(&lh, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
        if (e == cudaSuccess && grads)
            e = cudaMemcpyAsync(grads, g, (size_t)MLP_PARAMS * 4, cudaMemcpyDeviceToHost, n->stream);
        if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: copy out");
        rc = check_status(n, "st_mlp_loss_grad");
        if (rc) return rc;
        if (loss) *loss = (float)lh;
    }
    return ST_OK;
}

int st_track_surrogate(st_ctx* ctx, st_mlp* n, int32_t n_turns, double* spin_sum) {
    if (!ctx || !n) {
        set_error("st_track_surrogate: null pointer");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_track_surrogate: no particles uploaded");
        return ST_ESTATE;
    }
    if (n_turns < 0 || ctx->n > n->max_batch || ctx->precision != ST_FP64) {
        set_error("st_track_surrogate: need n_turns >= 0, n_particles <= the network's max_batch, FP64 context");
        return ST_EINVAL;
    }
    const int B = (int)ctx->n;
    const int Bp = ((B + 127) / 128) * 128;
    // the network runs on the context's stream
    cudaStream_t keep = n->stream;
    n->stream = ctx->stream;
    int rc = ST_OK;
    cudaError_t e = cudaMemsetAsync(n->status, 0, sizeof(int32_t), n->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "st_track_surrogate: status");
    for (int t = 0; t < n_turns && rc == ST_OK; ++t) {
        // one-turn map from the orbit at the fixed azimuth (start of the turn)
        mlp_pack_state<<<(Bp + 127) / 128, 128, 0, n->stream>>>(ctx->xpx, ctx->ypy, ctx->tpt, B, Bp, n->head, n->Xf,
                                                                n->X0);
        rc = mlp_forward_layers(n, Bp, false);
        if (rc) break;
        surrogate_apply<<<(B + 127) / 128, 128, 0, n->stream>>>(n->Y, n->Xf, B, n->head, ctx->sxy, ctx->sz, ctx->lost,
                                                                spin_sum);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "st_track_surrogate: spin step");
            break;
        }
        rc = launch_track_orbit(ctx, 1);
    }
    n->stream = keep;
    return rc;
}

int st_mlp_adam_step(st_mlp* n, float lr, float beta1, float beta2, float eps) {
    if (!n || !n->have_grads || !(lr > 0.0f)) {
        set_error("st_mlp_adam_step: no gradients or lr <= 0");
        return ST_EINVAL;
    }
    n->step += 1;
    const float c1 = 1.0f / (1.0f - powf(beta1, (float)n->step));
    const float c2 = 1.0f / (1.0f - powf(beta2, (float)n->step));
    const int64_t P = MLP_PARAMS;
    mlp_adam<<<(unsigned)((P + 255) / 256), 256, 0, n->stream>>>(n->p, n->m, n->v, n->g, P, lr, beta1, beta2, eps, c1,
                                                                 c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_adam_step");
    return mlp_refresh_weights(n);
}

}  // extern "C"
