// Learned one-turn spin map: a multilayer perceptron 6 -> 256 -> 256 -> 256 ->
// 256 -> 4 with SiLU activations whose layers run on the tcgen05 BF16 GEMM
// (gemm_bf16_tn: bf16 weights and activations, FP32 accumulation in tensor
// memory), FP32 master weights and Adam moments, and an FP64 head:
//
//     u = q0 + P(x) + s y,   q = u / |u|,   x = in_scale * z,
//
// q0 the closed-orbit one-turn quaternion, P a polynomial of degree <= 3 in x
// fitted by FP64 least squares over tracked pairs (degree 1 = a linear term),
// s the output scales (one per component) and y the network's 4 outputs.  The
// network learns the residual (q - q0 - P(x)) / s, component by component.
//
// The scaled input is handed to the first layer as two bf16 numbers (hi and
// the bf16 rounding of x - hi) multiplying the same weight column, so the
// network sees x to about 2^-16 relative although every operand is bf16; the
// first layer's K = 64 padding has room for both at no extra cost.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "st_internal.cuh"
#include "tc_gemm.cuh"

namespace st {

constexpr int MLP_IN = 6, MLP_H = 256, MLP_OUT = 4, MLP_KIN = 64, MLP_NOUT = 16;
constexpr int POLY_MAX_DEG = 3, POLY_MAX = 84;   // monomials of 6 inputs up to degree 3
constexpr int WG_MAX_SPLITS = 64;                 // split-K pieces of the weight-gradient GEMMs

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

// Monomials of the 6 inputs up to a degree, graded: 1; x0..x5; x_i x_j
// (i <= j, i outer); x_i x_j x_k (i <= j <= k).  Each is three input indices,
// 6 standing for "none".  Returns the count (1, 7, 28 or 84).
static int build_terms(int degree, uint8_t terms[POLY_MAX][3]) {
    int f = 0;
    terms[f][0] = terms[f][1] = terms[f][2] = MLP_IN;
    ++f;
    if (degree >= 1)
        for (int i = 0; i < MLP_IN; ++i, ++f) {
            terms[f][0] = (uint8_t)i;
            terms[f][1] = terms[f][2] = MLP_IN;
        }
    if (degree >= 2)
        for (int i = 0; i < MLP_IN; ++i)
            for (int j = i; j < MLP_IN; ++j, ++f) {
                terms[f][0] = (uint8_t)i;
                terms[f][1] = (uint8_t)j;
                terms[f][2] = MLP_IN;
            }
    if (degree >= 3)
        for (int i = 0; i < MLP_IN; ++i)
            for (int j = i; j < MLP_IN; ++j)
                for (int k = j; k < MLP_IN; ++k, ++f) {
                    terms[f][0] = (uint8_t)i;
                    terms[f][1] = (uint8_t)j;
                    terms[f][2] = (uint8_t)k;
                }
    return f;
}

// The FP64 head.  terms / coef point to device memory: terms [n_terms][3],
// coef [4][POLY_MAX]; one output scale per quaternion component.
struct PolyHead {
    double q0[4];
    double scale[4];
    double in_scale[MLP_IN];
    int32_t n_terms;
    const uint8_t* terms;
    const double* coef;
};

// input scales for the layout kernels
struct InScale {
    float s[MLP_IN];
};

}  // namespace st

struct st_mlp {
    int32_t max_batch = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __nv_bfloat16 *W1p = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr, *W5p = nullptr;
    __nv_bfloat16 *W2T = nullptr, *W3T = nullptr, *W4T = nullptr, *W5Tp = nullptr;
    __nv_bfloat16 *X0 = nullptr, *X0T = nullptr;            // [Bp][64] / [64][Bp]: hi, lo, zero
    __nv_bfloat16* A[4] = {nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16* AT[4] = {nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16* DS[4] = {nullptr, nullptr, nullptr, nullptr};   // SiLU'(z) of the hidden layers, [Bp][256]
    float* Y = nullptr;                                     // [Bp][16]
    __nv_bfloat16 *dYp = nullptr, *dYT = nullptr;
    __nv_bfloat16* dZ[2] = {nullptr, nullptr};
    __nv_bfloat16* dZT[2] = {nullptr, nullptr};
    float* dWtmp = nullptr;                                 // [256][64]
    float* ws = nullptr;                                    // split-K partial sums [64][256][256]
    float* b5p = nullptr;                                   // [16] output bias, zero padded
    double* loss = nullptr;
    int32_t* status = nullptr;
    uint8_t* d_terms = nullptr;                             // [POLY_MAX][3]
    double* d_coef = nullptr;                               // [4][POLY_MAX]
    double h_coef[4][st::POLY_MAX];
    uint8_t h_terms[st::POLY_MAX][3];
    int32_t degree = 1;
    st::PolyHead head;
    st::InScale in_scale;
    int64_t step = 0;
    bool have_grads = false;
    bool fused_inference = true;   // inference through the fused five-layer kernel
};

namespace st {

__device__ __forceinline__ void poly_eval(const PolyHead& h, const double* xs, double* out) {
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (int f = 0; f < h.n_terms; ++f) {
        double mono = 1.0;
        for (int j = 0; j < 3; ++j) {
            const int c = h.terms[3 * f + j];
            if (c < MLP_IN) mono *= xs[c];
        }
        for (int k = 0; k < 4; ++k) out[k] = fma(h.coef[k * POLY_MAX + f], mono, out[k]);
    }
}

// u = q0 + P(x) + s y in FP64
__device__ __forceinline__ void head_u(const PolyHead& h, const double* xs, const float* y, double* u) {
    double pv[4];
    poly_eval(h, xs, pv);
    for (int k = 0; k < 4; ++k) u[k] = h.q0[k] + pv[k] + h.scale[k] * (double)y[k];
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));   // v - hi is exact in FP32
}

// one row of the first layer's input: hi parts in columns 0..5, lo parts in
// 6..11, zeros after; the row-major copy is written as 16-byte vectors
__device__ __forceinline__ void write_input_row(const float* xs, int r, int Bp, __nv_bfloat16* __restrict__ X0,
                                                __nv_bfloat16* __restrict__ X0T) {
    __align__(16) __nv_bfloat16 row[16];
    for (int c = 0; c < MLP_IN; ++c) split_bf16(xs[c], row[c], row[MLP_IN + c]);
    row[12] = row[13] = row[14] = row[15] = __float2bfloat16_rn(0.0f);
    uint4* dst = reinterpret_cast<uint4*>(X0 + (size_t)r * MLP_KIN);
    dst[0] = *reinterpret_cast<const uint4*>(&row[0]);
    dst[1] = *reinterpret_cast<const uint4*>(&row[8]);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (int k = 2; k < MLP_KIN / 8; ++k) dst[k] = zero4;
    if (X0T)
        for (int c = 0; c < MLP_KIN; ++c)
            X0T[(size_t)c * Bp + r] = c < 16 ? row[c] : __float2bfloat16_rn(0.0f);
}

// rows, step (optional): the batch starts at row rows[*step] of x (a training
// schedule replayed from a CUDA graph)
__global__ void mlp_pack_x(const float* __restrict__ x, int B, int Bp, InScale is, __nv_bfloat16* __restrict__ X0,
                           __nv_bfloat16* __restrict__ X0T, const int64_t* __restrict__ rows = nullptr,
                           const int32_t* __restrict__ step = nullptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bp) return;
    if (rows) x += rows[*step] * MLP_IN;
    float xs[MLP_IN];
    for (int c = 0; c < MLP_IN; ++c) xs[c] = r < B ? x[(size_t)r * MLP_IN + c] * is.s[c] : 0.0f;
    write_input_row(xs, r, Bp, X0, X0T);
}

// the same from the tracker's FP64 pair-SoA state (coordinates X..Pt)
__global__ void mlp_pack_state(const double2* __restrict__ xpx, const double2* __restrict__ ypy,
                               const double2* __restrict__ tpt, int B, int Bp, PolyHead h,
                               __nv_bfloat16* __restrict__ X0) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bp) return;
    float xs[MLP_IN] = {0, 0, 0, 0, 0, 0};
    if (r < B) {
        const double2 a = xpx[r], b = ypy[r], c = tpt[r];
        const double z[MLP_IN] = {a.x, a.y, b.x, b.y, c.x, c.y};
        for (int k = 0; k < MLP_IN; ++k) xs[k] = (float)(z[k] * h.in_scale[k]);
    }
    write_input_row(xs, r, Bp, X0, nullptr);
}

// writes dL/dy (bf16, zero padded) row-major [Bp][64] and transposed [16][Bp]
__device__ __forceinline__ void write_dy(const float* gy, int r, int Bp, __nv_bfloat16* __restrict__ dYp,
                                         __nv_bfloat16* __restrict__ dYT) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(gy[0], gy[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(gy[2], gy[3]);
    uint4* dst = reinterpret_cast<uint4*>(dYp + (size_t)r * MLP_KIN);
    dst[0] = make_uint4(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b), 0u, 0u);
    for (int k = 1; k < MLP_KIN / 8; ++k) dst[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int c = 0; c < MLP_NOUT; ++c) dYT[(size_t)c * Bp + r] = __float2bfloat16_rn(c < 4 ? gy[c] : 0.0f);
}

// block sum of l, one double atomic per block
__device__ __forceinline__ void block_loss_add(double l, double* loss) {
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t);
    }
}

// Quaternion head: q = u / |u|; with targets the loss mean_b |q_b - qt_b|^2 and
// dL/dy = s (I - q q^T) (2 (q - qt) / B) / |u|.
__global__ void mlp_head_quat(const float* __restrict__ Y, const float* __restrict__ x, int B, int Bp, PolyHead h,
                              const float* __restrict__ qt, float* __restrict__ q_out, double* __restrict__ loss,
                              __nv_bfloat16* __restrict__ dYp, __nv_bfloat16* __restrict__ dYT) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (r < Bp) {
        float gy[4] = {0, 0, 0, 0};
        if (r < B) {
            double xs[MLP_IN], u[4];
            for (int c = 0; c < MLP_IN; ++c) xs[c] = (double)x[(size_t)r * MLP_IN + c] * h.in_scale[c];
            head_u(h, xs, Y + (size_t)r * MLP_NOUT, u);
            const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
            double q[4];
            for (int k = 0; k < 4; ++k) q[k] = u[k] / nu;
            if (q_out)
                for (int k = 0; k < 4; ++k) q_out[(size_t)r * 4 + k] = (float)q[k];
            if (qt) {
                double d[4], dq = 0.0;
                for (int k = 0; k < 4; ++k) {
                    d[k] = q[k] - (double)qt[(size_t)r * 4 + k];
                    l += d[k] * d[k];
                    dq += q[k] * d[k];
                }
                for (int k = 0; k < 4; ++k) gy[k] = (float)(h.scale[k] * (2.0 / B) * (d[k] - q[k] * dq) / nu);
            }
        }
        if (dYp) write_dy(gy, r, Bp, dYp, dYT);
    }
    if (loss) block_loss_add(l / B, loss);
}

// Residual head: loss mean_b |y_b - r_b|^2, dL/dy = 2 (y - r) / B.
__global__ void mlp_head_resid(const float* __restrict__ Y, const float* __restrict__ rt, int B, int Bp,
                               double* __restrict__ loss, __nv_bfloat16* __restrict__ dYp,
                               __nv_bfloat16* __restrict__ dYT, const int64_t* __restrict__ rows = nullptr,
                               const int32_t* __restrict__ step = nullptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (rows) rt += rows[*step] * MLP_OUT;
    double l = 0.0;
    if (r < Bp) {
        float gy[4] = {0, 0, 0, 0};
        if (r < B) {
            for (int k = 0; k < 4; ++k) {
                const float d = Y[(size_t)r * MLP_NOUT + k] - rt[(size_t)r * 4 + k];
                l += (double)d * d;
                gy[k] = (2.0f / B) * d;
            }
        }
        write_dy(gy, r, Bp, dYp, dYT);
    }
    block_loss_add(l / B, loss);
}

// end of a replayed training step: record its loss, advance the step counter
__global__ void mlp_step_end(int32_t* __restrict__ step, const double* __restrict__ loss, double* __restrict__ losses) {
    if (losses) losses[*step] = *loss;
    *step += 1;
}

// row sums of a [rows][Bp] bf16 matrix (bias gradients): one block of 256
// threads per row, 16-byte loads of 8 values (Bp is a multiple of 128, rows
// 16-byte aligned), a fixed-order tree over the block
constexpr int ROWSUM_THREADS = 256;
__global__ void __launch_bounds__(ROWSUM_THREADS) mlp_rowsum(const __nv_bfloat16* __restrict__ M, int rows, int Bp,
                                                            float* __restrict__ out) {
    __shared__ float red[ROWSUM_THREADS / 32];
    const int row = blockIdx.x;
    const uint4* v = reinterpret_cast<const uint4*>(M + (size_t)row * Bp);
    const int n8 = Bp / 8;
    float s = 0.0f;
#pragma unroll 4
    for (int c = threadIdx.x; c < n8; c += ROWSUM_THREADS) {
        const uint4 q = v[c];
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            s += f.x + f.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < ROWSUM_THREADS / 32; ++k) t += red[k];
        if (row < rows) out[row] = t;
    }
}

// dW1 [256][6] from dWtmp [256][64]: the hi and lo input columns share W1
__global__ void mlp_gather_w1(const float* __restrict__ tmp, float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_H * MLP_IN) return;
    const int r = i / MLP_IN, c = i % MLP_IN;
    g[i] = tmp[r * MLP_KIN + c] + tmp[r * MLP_KIN + MLP_IN + c];
}
// dW5 [4][256] from D' [256][16] (transposed)
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
    // W1p [256][64]: W1 in columns 0..5 (hi inputs) and again in 6..11 (lo inputs)
    if (i < MLP_H * MLP_KIN) {
        const int r = i / MLP_KIN, c = i % MLP_KIN;
        W1p[i] = __float2bfloat16_rn(c < 2 * MLP_IN ? p[mlp_w_off(0) + r * MLP_IN + c % MLP_IN] : 0.0f);
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

// sched, step (optional): lr, c1, c2 of step *step from sched[3 step ...]
__global__ void mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                         const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                         float c2, const float* __restrict__ sched = nullptr, const int32_t* __restrict__ step = nullptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (sched) {
        const int s = *step;
        lr = sched[3 * s];
        c1 = sched[3 * s + 1];
        c2 = sched[3 * s + 2];
    }
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Spin step of the learned map: q = normalise(q0 + P(x) + s y) in FP64 from
// the FP64 orbit at s = 0 and the FP32 network output, S <- q S conj(q);
// optional running sum of S.
__global__ void surrogate_apply(const float* __restrict__ Y, int B, PolyHead h, const double2* __restrict__ xpx,
                                const double2* __restrict__ ypy, const double2* __restrict__ tpt,
                                double2* __restrict__ sxy, double* __restrict__ szp, const uint8_t* __restrict__ lost,
                                double* __restrict__ sum) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B || lost[r]) return;
    const double2 a = xpx[r], b = ypy[r], c = tpt[r];
    const double z[MLP_IN] = {a.x, a.y, b.x, b.y, c.x, c.y};
    double xs[MLP_IN], u[4];
    for (int k = 0; k < MLP_IN; ++k) xs[k] = z[k] * h.in_scale[k];
    head_u(h, xs, Y + (size_t)r * MLP_NOUT, u);
    Quat q = qnormalize(Quat{u[0], u[1], u[2], u[3]});
    const double2 s2 = sxy[r];
    double sx = s2.x, sy = s2.y, sz = szp[r];
    rotate_vec(q, sx, sy, sz);
    sxy[r] = make_double2(sx, sy);
    szp[r] = sz;
    if (sum) {
        sum[r] += sx;
        sum[(size_t)B + r] += sy;
        sum[2 * (size_t)B + r] += sz;
    }
}

// Training rows from the tracker's SoA FP64 pairs (z [6][n] before the turn,
// q [4][n] its one-turn quaternion): x_rows = z (float), r_rows = the residual
// target (q - q0 - P(x)) / s (computed in FP64, stored as float).
__global__ void mlp_make_targets(const double* __restrict__ z, const double* __restrict__ q, int64_t n, PolyHead h,
                                 float* __restrict__ x_rows, float* __restrict__ r_rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xs[MLP_IN], pv[4];
    for (int c = 0; c < MLP_IN; ++c) {
        const double zc = z[c * n + i];
        x_rows[i * MLP_IN + c] = (float)zc;
        xs[c] = zc * h.in_scale[c];
    }
    poly_eval(h, xs, pv);
    for (int k = 0; k < 4; ++k) r_rows[i * 4 + k] = (float)((q[k * n + i] - h.q0[k] - pv[k]) / h.scale[k]);
}

// FP64 moments of the least-squares fit q - q0 ~ P(x): with features f (the
// n_terms monomials) and responses e = q - q0, the products f_a f_b (a <= b),
// f_a e_k and e_k e_k summed over the pairs, one value per entry of the pair
// table (pa, pb index the row [f, e]).  Rows are staged 32 at a time in shared
// memory; each thread owns up to FIT_PER_THREAD table entries.
constexpr int FIT_ROWS = 32, FIT_THREADS = 256, FIT_PER_THREAD = 16;
constexpr int FIT_W = POLY_MAX + 4;

__global__ void __launch_bounds__(FIT_THREADS) mlp_fit_moments(const double* __restrict__ z,
                                                               const double* __restrict__ q,
                                                               const uint8_t* __restrict__ lost, int64_t n,
                                                               PolyHead h, const uint8_t* __restrict__ pa,
                                                               const uint8_t* __restrict__ pb, int n_entries,
                                                               double* __restrict__ mom) {
    __shared__ double rows[FIT_ROWS][FIT_W];
    const int F = h.n_terms, W = F + 4;
    double acc[FIT_PER_THREAD];
    int ea[FIT_PER_THREAD], eb[FIT_PER_THREAD];
#pragma unroll
    for (int o = 0; o < FIT_PER_THREAD; ++o) {
        acc[o] = 0.0;
        const int t = threadIdx.x + o * FIT_THREADS;
        ea[o] = t < n_entries ? pa[t] : 0;
        eb[o] = t < n_entries ? pb[t] : 0;
    }
    const int64_t n_chunks = (n + FIT_ROWS - 1) / FIT_ROWS;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        for (int e = threadIdx.x; e < FIT_ROWS * W; e += FIT_THREADS) {
            const int row = e / W, col = e % W;
            const int64_t i = ch * FIT_ROWS + row;
            double val = 0.0;
            if (i < n && !(lost && lost[i])) {
                if (col < F) {
                    val = 1.0;
                    for (int j = 0; j < 3; ++j) {
                        const int c = h.terms[3 * col + j];
                        if (c < MLP_IN) val *= z[c * n + i] * h.in_scale[c];
                    }
                } else {
                    val = q[(col - F) * n + i] - h.q0[col - F];
                }
            }
            rows[row][col] = val;
        }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < FIT_PER_THREAD; ++o) {
            if (threadIdx.x + o * FIT_THREADS < n_entries) {
                double s = acc[o];
                for (int row = 0; row < FIT_ROWS; ++row) s = fma(rows[row][ea[o]], rows[row][eb[o]], s);
                acc[o] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 0; o < FIT_PER_THREAD; ++o) {
        const int t = threadIdx.x + o * FIT_THREADS;
        if (t < n_entries) atomicAdd(&mom[t], acc[o]);
    }
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

static int upload_head(st_mlp* n) {
    cudaError_t e = cudaMemcpyAsync(n->d_coef, n->h_coef, sizeof(n->h_coef), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->d_terms, n->h_terms, sizeof(n->h_terms), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "mlp: head upload");
}

// forward through the five layers from X0 (rows Bp); keep_t writes the
// transposed activations and the SiLU derivatives (bf16) for a following
// backward pass
static int mlp_forward_layers(st_mlp* n, int Bp, bool keep_t) {
    if (!keep_t && n->fused_inference) {
        // inference: all five layers per 128-row tile in one kernel
        const void* W[5] = {n->W1p, n->W2, n->W3, n->W4, n->W5p};
        const float* b[5] = {n->p + mlp_b_off(0), n->p + mlp_b_off(1), n->p + mlp_b_off(2), n->p + mlp_b_off(3),
                             n->b5p};
        return mlp_fused_forward(n->X0, W, b, n->Y, Bp, n->status, n->stream);
    }
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
        e.ds_out = keep_t ? n->DS[l] : nullptr;
        e.ld_dso = MLP_H;
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

// Weight gradient out[M][N] = A . B^T with the batch as K (K = Bp): few
// output tiles and a long K, so K is split across CTAs and the partial sums
// reduced (deterministic order).
static int wgrad_gemm(st_mlp* n, const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int Bp, float* out,
                      cudaStream_t stream) {
    GemmEpi ep = epi_base();
    ep.mode = EPI_F32;
    ep.n_valid = N;
    ep.ld_f32 = N;
    const int splits = gemm_split_count(Bp, WG_MAX_SPLITS);
    if (splits == 1) {
        ep.out_f32 = out;
        return gemm_bf16_tn(A, B, M, N, Bp, ep, n->status, stream);
    }
    ep.out_f32 = n->ws;
    ep.split_stride = (int64_t)M * N;
    int rc = gemm_bf16_tn(A, B, M, N, Bp, ep, n->status, stream, splits);
    if (rc) return rc;
    return gemm_split_reduce(n->ws, splits, (int64_t)M * N, (int64_t)M * N, out, stream);
}

// Streams of a backward pass: the data gradients (the chain to the next layer)
// on `main`; the weight gradients of each layer, which only the optimiser
// reads, on `side` and its bias gradients on `side2` when they are given (a
// captured training step),
// forked after the data gradient they read and joined back at the end.  The
// data gradient of layer l - 1 overwrites the buffer that layer l + 1's weight
// gradient reads, so it waits for that one.  The kernels and their order on
// each stream are those of the single-stream pass, so the results are equal.
struct BackwardStreams {
    cudaStream_t main, side, side2;   // side2: the bias-gradient row sums
    cudaEvent_t fork, done, join, done2, join2;
};

static int bw_event(cudaError_t e, const char* what) { return e == cudaSuccess ? ST_OK : cuda_fail(e, what); }

// Backward pass from dL/dy (dYp, dYT written by a head kernel) into the
// gradient buffer g, using the activations kept by the forward pass.
static int mlp_backward(st_mlp* n, int Bp, const BackwardStreams* bs = nullptr) {
    float* g = n->g;
    const cudaStream_t ms = n->stream, ss = bs ? bs->side : n->stream, s2 = bs ? bs->side2 : n->stream;
    auto fork = [&]() -> int {   // the side streams wait for the main stream's work so far
        if (!bs) return ST_OK;
        int rc = bw_event(cudaEventRecord(bs->fork, ms), "mlp: backward fork");
        if (!rc) rc = bw_event(cudaStreamWaitEvent(ss, bs->fork, 0), "mlp: backward fork");
        return rc ? rc : bw_event(cudaStreamWaitEvent(s2, bs->fork, 0), "mlp: backward fork");
    };
    auto side_done = [&]() -> int {
        if (!bs) return ST_OK;
        int rc = bw_event(cudaEventRecord(bs->done, ss), "mlp: backward side");
        return rc ? rc : bw_event(cudaEventRecord(bs->done2, s2), "mlp: backward side");
    };
    auto wait_side = [&]() -> int {   // the main stream waits for the side work recorded last
        if (!bs) return ST_OK;
        int rc = bw_event(cudaStreamWaitEvent(ms, bs->done, 0), "mlp: backward wait");
        return rc ? rc : bw_event(cudaStreamWaitEvent(ms, bs->done2, 0), "mlp: backward wait");
    };
    // layer 5: dW5^T = A4^T . dY  (D'[256][16]), db5 = sum dY, dZ4 = (dY W5) * silu'(Z4)
    int rc = fork();
    if (!rc) rc = wgrad_gemm(n, n->AT[3], n->dYT, MLP_H, MLP_NOUT, Bp, n->dWtmp, ss);
    if (rc) return rc;
    mlp_gather_w5<<<(MLP_OUT * MLP_H + 255) / 256, 256, 0, ss>>>(n->dWtmp, g + mlp_w_off(4));
    mlp_rowsum<<<MLP_OUT, ROWSUM_THREADS, 0, s2>>>(n->dYT, MLP_OUT, Bp, g + mlp_b_off(4));
    if ((rc = side_done())) return rc;
    GemmEpi ep = epi_base();
    ep.mode = EPI_DSILU;
    ep.n_valid = MLP_H;
    ep.ds_in = n->DS[3];
    ep.ld_ds = MLP_H;
    ep.out_bf16 = n->dZ[0];
    ep.ld_bf16 = MLP_H;
    ep.out_bf16_t = n->dZT[0];
    ep.ld_bf16_t = Bp;
    rc = gemm_bf16_tn(n->dYp, n->W5Tp, Bp, MLP_H, MLP_KIN, ep, n->status, ms);
    if (rc) return rc;
    // hidden layers l = 3, 2, 1 (0-based weights W[l], activations A[l-1])
    const __nv_bfloat16* WT[4] = {nullptr, n->W2T, n->W3T, n->W4T};
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        // dW_l = dZ_l^T . A_{l-1}  ->  [256 out][256 in], into the gradient buffer
        if ((rc = fork())) return rc;
        // (the main stream's next data gradient overwrites what the previous
        // iteration's side work reads: wait for it first)
        if (l < 3 && (rc = wait_side())) return rc;
        rc = wgrad_gemm(n, n->dZT[cur], n->AT[l - 1], MLP_H, MLP_H, Bp, g + mlp_w_off(l), ss);
        if (rc) return rc;
        mlp_rowsum<<<MLP_H, ROWSUM_THREADS, 0, s2>>>(n->dZT[cur], MLP_H, Bp, g + mlp_b_off(l));
        if ((rc = side_done())) return rc;
        // dZ_{l-1} = (dZ_l W_l) * silu'(Z_{l-1})
        ep = epi_base();
        ep.mode = EPI_DSILU;
        ep.n_valid = MLP_H;
        ep.ds_in = n->DS[l - 1];
        ep.ld_ds = MLP_H;
        ep.out_bf16 = n->dZ[1 - cur];
        ep.ld_bf16 = MLP_H;
        ep.out_bf16_t = n->dZT[1 - cur];
        ep.ld_bf16_t = Bp;
        rc = gemm_bf16_tn(n->dZ[cur], WT[l], Bp, MLP_H, MLP_H, ep, n->status, ms);
        if (rc) return rc;
        cur = 1 - cur;
    }
    // layer 1: dW1 = dZ1^T . X0 -> [256][64] -> [256][6] (hi + lo columns); db1
    if ((rc = fork())) return rc;
    rc = wgrad_gemm(n, n->dZT[cur], n->X0T, MLP_H, MLP_KIN, Bp, n->dWtmp, ss);
    if (rc) return rc;
    mlp_gather_w1<<<(MLP_H * MLP_IN + 255) / 256, 256, 0, ss>>>(n->dWtmp, g + mlp_w_off(0));
    mlp_rowsum<<<MLP_H, ROWSUM_THREADS, 0, s2>>>(n->dZT[cur], MLP_H, Bp, g + mlp_b_off(0));
    if (bs) {   // join: the main stream continues after all the gradients
        if ((rc = bw_event(cudaEventRecord(bs->join, ss), "mlp: backward join"))) return rc;
        if ((rc = bw_event(cudaEventRecord(bs->join2, s2), "mlp: backward join"))) return rc;
        if ((rc = bw_event(cudaStreamWaitEvent(ms, bs->join, 0), "mlp: backward join"))) return rc;
        if ((rc = bw_event(cudaStreamWaitEvent(ms, bs->join2, 0), "mlp: backward join"))) return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp: backward");
    n->have_grads = true;
    return ST_OK;
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

// loss / gradient copies to the host (optional), then the status check
static int finish_loss_grad(st_mlp* n, float* loss, float* grads, const char* what) {
    if (!loss && !grads) return ST_OK;
    double lh = 0.0;
    cudaError_t e = cudaSuccess;
    if (loss) e = cudaMemcpyAsync(&lh, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess && grads)
        e = cudaMemcpyAsync(grads, n->g, (size_t)MLP_PARAMS * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    int rc = check_status(n, what);
    if (rc) return rc;
    if (loss) *loss = (float)lh;
    return ST_OK;
}

static int check_batch(st_mlp* n, const void* x, const void* t, int32_t B, const char* what) {
    if (!n || !x || !t || B < 1 || B > n->max_batch) {
        set_error("%s: null pointer or batch outside 1..max_batch", what);
        return ST_EINVAL;
    }
    return ST_OK;
}

}  // namespace st

using namespace st;

extern "C" {

int64_t st_mlp_param_count(void) { return MLP_PARAMS; }

int st_mlp_destroy(st_mlp* n) {
    if (!n) return ST_OK;
    cudaStreamSynchronize(n->stream);
    void* ptrs[] = {n->p,   n->m,   n->v,   n->g,   n->W1p, n->W2,  n->W3,   n->W4,      n->W5p,  n->W2T,
                    n->W3T, n->W4T, n->W5Tp, n->X0, n->X0T, n->Y,   n->dYp,  n->dYT,     n->dWtmp, n->ws, n->b5p,
                    n->loss, n->status, n->d_terms, n->d_coef};
    for (void* q : ptrs) cudaFree(q);
    for (int l = 0; l < 4; ++l) {
        cudaFree(n->A[l]);
        cudaFree(n->AT[l]);
        cudaFree(n->DS[l]);
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
    ST_MALLOC(n->X0, (size_t)Bp * MLP_KIN * bf);
    ST_MALLOC(n->X0T, (size_t)Bp * MLP_KIN * bf);
    for (int l = 0; l < 4; ++l) {
        ST_MALLOC(n->A[l], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->AT[l], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->DS[l], (size_t)Bp * MLP_H * 2);
    }
    ST_MALLOC(n->Y, (size_t)Bp * MLP_NOUT * 4);
    ST_MALLOC(n->dYp, (size_t)Bp * MLP_KIN * bf);
    ST_MALLOC(n->dYT, (size_t)Bp * MLP_NOUT * bf);
    for (int k = 0; k < 2; ++k) {
        ST_MALLOC(n->dZ[k], (size_t)Bp * MLP_H * bf);
        ST_MALLOC(n->dZT[k], (size_t)Bp * MLP_H * bf);
    }
    ST_MALLOC(n->dWtmp, (size_t)MLP_H * MLP_KIN * 4);
    ST_MALLOC(n->ws, (size_t)WG_MAX_SPLITS * MLP_H * MLP_H * 4);
    ST_MALLOC(n->b5p, MLP_NOUT * 4);
    ST_MALLOC(n->loss, sizeof(double));
    ST_MALLOC(n->status, sizeof(int32_t));
    ST_MALLOC(n->d_terms, sizeof(n->h_terms));
    ST_MALLOC(n->d_coef, sizeof(n->h_coef));
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
    // head: q0 = 1, no polynomial, s = 1, unit input scales
    memset(n->h_coef, 0, sizeof(n->h_coef));
    memset(&n->head, 0, sizeof(n->head));
    n->degree = 1;
    n->head.n_terms = build_terms(1, n->h_terms);
    n->head.q0[0] = 1.0;
    for (int k = 0; k < 4; ++k) n->head.scale[k] = 1.0;
    for (int c = 0; c < MLP_IN; ++c) {
        n->head.in_scale[c] = 1.0;
        n->in_scale.s[c] = 1.0f;
    }
    n->head.terms = n->d_terms;
    n->head.coef = n->d_coef;
    int rc = upload_head(n);
    if (rc == ST_OK) rc = mlp_refresh_weights(n);
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
    for (int c = 0; c < MLP_IN; ++c)
        if (!(in_scale[c] >= 0.0) || !std::isfinite(in_scale[c])) {
            set_error("st_mlp_set_head: input scales must be finite and >= 0");
            return ST_EINVAL;
        }
    memset(n->h_coef, 0, sizeof(n->h_coef));
    n->degree = 1;
    n->head.n_terms = build_terms(1, n->h_terms);
    for (int k = 0; k < 4; ++k) {
        n->head.q0[k] = q0[k];
        for (int c = 0; c < MLP_IN; ++c) n->h_coef[k][1 + c] = lin ? lin[k * MLP_IN + c] : 0.0;
    }
    for (int k = 0; k < 4; ++k) n->head.scale[k] = out_scale;
    for (int c = 0; c < MLP_IN; ++c) {
        n->head.in_scale[c] = in_scale[c];
        n->in_scale.s[c] = (float)in_scale[c];
    }
    return upload_head(n);
}

int st_mlp_set_scale(st_mlp* n, const double* out_scale) {
    if (!n || !out_scale) {
        set_error("st_mlp_set_scale: null pointer");
        return ST_EINVAL;
    }
    for (int k = 0; k < 4; ++k)
        if (!(out_scale[k] > 0.0) || !std::isfinite(out_scale[k])) {
            set_error("st_mlp_set_scale: need finite output scales > 0");
            return ST_EINVAL;
        }
    for (int k = 0; k < 4; ++k) n->head.scale[k] = out_scale[k];
    return ST_OK;
}

int st_mlp_fit_head(st_mlp* nw, int32_t degree, const double* z_soa, const double* q_soa, const uint8_t* lost,
                    int64_t n, double* coef_out, double* rms_out) {
    if (!nw || !z_soa || !q_soa || n < 1 || degree < 0 || degree > POLY_MAX_DEG) {
        set_error("st_mlp_fit_head: null pointer, n < 1 or degree outside 0..3");
        return ST_EINVAL;
    }
    uint8_t terms[POLY_MAX][3];
    const int F = build_terms(degree, terms);
    // table of products: f_a f_b (a <= b), f_a e_k, e_k e_k
    static_assert(POLY_MAX * (POLY_MAX + 1) / 2 + 4 * POLY_MAX + 4 <= FIT_THREADS * FIT_PER_THREAD, "fit table");
    uint8_t pa[FIT_THREADS * FIT_PER_THREAD], pb[FIT_THREADS * FIT_PER_THREAD];
    int T = 0;
    for (int a = 0; a < F; ++a)
        for (int b = a; b < F; ++b, ++T) {
            pa[T] = (uint8_t)a;
            pb[T] = (uint8_t)b;
        }
    const int h_off = T;
    for (int a = 0; a < F; ++a)
        for (int k = 0; k < 4; ++k, ++T) {
            pa[T] = (uint8_t)a;
            pb[T] = (uint8_t)(F + k);
        }
    const int r_off = T;
    for (int k = 0; k < 4; ++k, ++T) pa[T] = pb[T] = (uint8_t)(F + k);

    memcpy(nw->h_terms, terms, sizeof(terms));
    nw->head.n_terms = F;
    int rc = upload_head(nw);   // the kernel reads the new monomial table
    if (rc) return rc;
    uint8_t* d_tab = nullptr;
    double* d_mom = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_tab, 2 * (size_t)T, nw->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_mom, (size_t)T * sizeof(double), nw->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, pa, T, cudaMemcpyHostToDevice, nw->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab + T, pb, T, cudaMemcpyHostToDevice, nw->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_mom, 0, (size_t)T * sizeof(double), nw->stream);
    std::vector<double> mom(FIT_THREADS * FIT_PER_THREAD, 0.0);
    if (e == cudaSuccess) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (n + FIT_ROWS - 1) / FIT_ROWS;
        if (blocks > 4 * sms) blocks = 4 * sms;
        mlp_fit_moments<<<(unsigned)blocks, FIT_THREADS, 0, nw->stream>>>(z_soa, q_soa, lost, n, nw->head, d_tab,
                                                                         d_tab + T, T, d_mom);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mom.data(), d_mom, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, nw->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nw->stream);
    cudaFreeAsync(d_tab, nw->stream);
    cudaFreeAsync(d_mom, nw->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_fit_head");

    // Normal equations over the monomials with nonzero sum of squares (an
    // input scale of 0 removes every monomial of its coordinate), solved by
    // Cholesky in FP64.
    std::vector<double> Gv((size_t)F * F), Cv((size_t)F * F, 0.0);
    auto G = [&](int a, int b) -> double& { return Gv[(size_t)a * F + b]; };
    auto C = [&](int a, int b) -> double& { return Cv[(size_t)a * F + b]; };
    int t = 0;
    for (int a = 0; a < F; ++a)
        for (int b = a; b < F; ++b, ++t) G(a, b) = G(b, a) = mom[t];
    int idx[POLY_MAX], m = 0;
    for (int a = 0; a < F; ++a)
        if (G(a, a) > 0.0) idx[m++] = a;
    for (int a = 0; a < m; ++a) {
        for (int b = 0; b <= a; ++b) {
            double s = G(idx[a], idx[b]);
            for (int c = 0; c < b; ++c) s -= C(a, c) * C(b, c);
            if (a == b) {
                if (!(s > 1e-300)) {
                    set_error("st_mlp_fit_head: singular normal equations (too few distinct pairs?)");
                    return ST_EINVAL;
                }
                C(a, a) = sqrt(s);
            } else {
                C(a, b) = s / C(b, b);
            }
        }
    }
    const double count = G(0, 0);
    double coef[4][POLY_MAX];
    memset(coef, 0, sizeof(coef));
    for (int k = 0; k < 4; ++k) {
        double y[POLY_MAX], sol[POLY_MAX];
        for (int a = 0; a < m; ++a) {
            double s = mom[h_off + idx[a] * 4 + k];
            for (int c = 0; c < a; ++c) s -= C(a, c) * y[c];
            y[a] = s / C(a, a);
        }
        for (int a = m - 1; a >= 0; --a) {
            double s = y[a];
            for (int c = a + 1; c < m; ++c) s -= C(c, a) * sol[c];
            sol[a] = s / C(a, a);
        }
        double rss = mom[r_off + k];
        for (int a = 0; a < m; ++a) {
            coef[k][idx[a]] = sol[a];
            rss -= sol[a] * mom[h_off + idx[a] * 4 + k];
        }
        if (rms_out) rms_out[k] = sqrt(rss > 0.0 ? rss / count : 0.0);
    }
    memset(nw->h_coef, 0, sizeof(nw->h_coef));
    for (int k = 0; k < 4; ++k)
        for (int f = 0; f < F; ++f) {
            nw->h_coef[k][f] = coef[k][f];
            if (coef_out) coef_out[k * F + f] = coef[k][f];
        }
    nw->degree = degree;
    return upload_head(nw);
}

int st_mlp_make_targets(st_mlp* nw, const double* z_soa, const double* q_soa, int64_t n, float* x_rows,
                        float* r_rows) {
    if (!nw || !z_soa || !q_soa || !x_rows || !r_rows || n < 1) {
        set_error("st_mlp_make_targets: null pointer or n < 1");
        return ST_EINVAL;
    }
    mlp_make_targets<<<(unsigned)((n + 255) / 256), 256, 0, nw->stream>>>(z_soa, q_soa, n, nw->head, x_rows, r_rows);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_make_targets");
}

int st_mlp_forward(st_mlp* n, const float* x, int32_t B, float* q_out) {
    int rc = check_batch(n, x, q_out, B, "st_mlp_forward");
    if (rc) return rc;
    const int Bp = ((B + 127) / 128) * 128;
    mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x, B, Bp, n->in_scale, n->X0, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_forward: pack");
    rc = mlp_forward_layers(n, Bp, false);
    if (rc) return rc;
    mlp_head_quat<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, x, B, Bp, n->head, nullptr, q_out, nullptr, nullptr,
                                                           nullptr);
    e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_forward: head");
}

int st_mlp_loss_grad(st_mlp* n, const float* x, const float* q_target, int32_t B, float* loss, float* grads) {
    int rc = check_batch(n, x, q_target, B, "st_mlp_loss_grad");
    if (rc) return rc;
    const int Bp = ((B + 127) / 128) * 128;
    cudaError_t e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: reset");
    mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x, B, Bp, n->in_scale, n->X0, n->X0T);
    rc = mlp_forward_layers(n, Bp, true);
    if (rc) return rc;
    mlp_head_quat<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, x, B, Bp, n->head, q_target, nullptr, n->loss,
                                                           n->dYp, n->dYT);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad: head");
    rc = mlp_backward(n, Bp);
    if (rc) return rc;
    return finish_loss_grad(n, loss, grads, "st_mlp_loss_grad");
}

int st_mlp_loss_grad_residual(st_mlp* n, const float* x, const float* r_target, int32_t B, float* loss,
                              float* grads) {
    int rc = check_batch(n, x, r_target, B, "st_mlp_loss_grad_residual");
    if (rc) return rc;
    const int Bp = ((B + 127) / 128) * 128;
    cudaError_t e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad_residual: reset");
    mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x, B, Bp, n->in_scale, n->X0, n->X0T);
    rc = mlp_forward_layers(n, Bp, true);
    if (rc) return rc;
    mlp_head_resid<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, r_target, B, Bp, n->loss, n->dYp, n->dYT);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "st_mlp_loss_grad_residual: head");
    rc = mlp_backward(n, Bp);
    if (rc) return rc;
    return finish_loss_grad(n, loss, grads, "st_mlp_loss_grad_residual");
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

int st_mlp_set_fused_inference(st_mlp* n, int32_t on) {
    if (!n) {
        set_error("st_mlp_set_fused_inference: null network");
        return ST_EINVAL;
    }
    n->fused_inference = on != 0;
    return ST_OK;
}

// Steps 1..steps-1 of a training schedule as one captured CUDA graph of a step
// (pack, forward, head, backward, Adam, weight refresh, step end) replayed
// once per step: the batch's rows and (lr, c1, c2) come from device arrays
// indexed by a device step counter, so every replay is the same graph.  The
// kernels and their arguments are those of the eager step, so the results
// are identical to stepping eagerly.
static int train_replayed(st_mlp* n, const float* x_rows, const float* r_rows, int32_t B, int32_t steps,
                          const int64_t* row_start, const float* lr, float beta1, float beta2, float eps,
                          double* d_loss) {
    const int Bp = ((B + 127) / 128) * 128;
    std::vector<float> sched(3 * (size_t)steps, 0.0f);
    for (int k = 1; k < steps; ++k) {
        // Adam's bias corrections at the optimiser step this schedule step makes
        const float t = (float)(n->step + k);
        sched[3 * k] = lr[k];
        sched[3 * k + 1] = 1.0f / (1.0f - powf(beta1, t));
        sched[3 * k + 2] = 1.0f / (1.0f - powf(beta2, t));
    }
    int64_t* d_rows = nullptr;
    float* d_sched = nullptr;
    int32_t* d_step = nullptr;
    const int32_t first = 1;
    cudaError_t e = cudaMallocAsync((void**)&d_rows, (size_t)steps * sizeof(int64_t), n->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_sched, sched.size() * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_step, sizeof(int32_t), n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_rows, row_start, (size_t)steps * sizeof(int64_t), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sched, sched.data(), sched.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_step, &first, sizeof(int32_t), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);   // the host arrays are transient
    int rc = e == cudaSuccess ? ST_OK : cuda_fail(e, "st_mlp_train: schedule upload");
    // capture and replay on a stream of our own (the caller's may be the legacy
    // default stream, which cannot be captured), joined to the caller's by events
    // (the weight gradients on a second stream, see mlp_backward)
    cudaStream_t caller = n->stream, cs = nullptr, side = nullptr, side2 = nullptr;
    cudaEvent_t ev = nullptr, evs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    if (rc == ST_OK) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&side2, cudaStreamNonBlocking);
        for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&evs[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, caller);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: replay stream");
    }
    if (rc == ST_OK) n->stream = cs;   // the step's launches go to the capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (rc == ST_OK) {
        e = cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: capture");
    }
    if (rc == ST_OK) {
        e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: loss reset");
        if (rc == ST_OK) {
            mlp_pack_x<<<(Bp + 127) / 128, 128, 0, n->stream>>>(x_rows, B, Bp, n->in_scale, n->X0, n->X0T, d_rows,
                                                                d_step);
            rc = mlp_forward_layers(n, Bp, true);
        }
        if (rc == ST_OK) {
            mlp_head_resid<<<(Bp + 127) / 128, 128, 0, n->stream>>>(n->Y, r_rows, B, Bp, n->loss, n->dYp, n->dYT,
                                                                    d_rows, d_step);
            const BackwardStreams bs{cs, side, side2, evs[0], evs[1], evs[2], evs[3], evs[4]};
            rc = mlp_backward(n, Bp, &bs);
        }
        if (rc == ST_OK) {
            const int64_t P = MLP_PARAMS;
            mlp_adam<<<(unsigned)((P + 255) / 256), 256, 0, n->stream>>>(n->p, n->m, n->v, n->g, P, 0.0f, beta1,
                                                                         beta2, eps, 0.0f, 0.0f, d_sched, d_step);
            rc = mlp_refresh_weights(n);
        }
        if (rc == ST_OK) mlp_step_end<<<1, 1, 0, n->stream>>>(d_step, n->loss, d_loss);
        const cudaError_t ec = cudaStreamEndCapture(n->stream, &graph);   // always end the capture
        if (rc == ST_OK && ec != cudaSuccess) rc = cuda_fail(ec, "st_mlp_train: capture");
    }
    if (rc == ST_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: graph instantiation");
    }
    for (int k = 1; k < steps && rc == ST_OK; ++k) {
        e = cudaGraphLaunch(exec, n->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: graph launch");
    }
    if (rc == ST_OK) n->step += steps - 1;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) {   // join the replays back into the caller's stream
        n->stream = caller;
        if (cudaEventRecord(ev, cs) == cudaSuccess) cudaStreamWaitEvent(caller, ev, 0);
        cudaStreamDestroy(cs);   // released once its work is done
    }
    if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t x : evs)
        if (x) cudaEventDestroy(x);
    if (side) cudaStreamDestroy(side);
    if (side2) cudaStreamDestroy(side2);
    cudaFreeAsync(d_rows, caller);
    cudaFreeAsync(d_sched, caller);
    cudaFreeAsync(d_step, caller);
    return rc;
}

int st_mlp_train(st_mlp* n, const float* x_rows, const float* r_rows, int64_t n_rows, int32_t B, int32_t steps,
                 const int64_t* row_start, const float* lr, float beta1, float beta2, float eps, double* loss_out) {
    if (!n || !x_rows || !r_rows || !row_start || !lr || steps < 0 || B < 1 || B > n->max_batch) {
        set_error("st_mlp_train: null pointer, steps < 0 or batch outside 1..max_batch");
        return ST_EINVAL;
    }
    for (int k = 0; k < steps; ++k)
        if (row_start[k] < 0 || row_start[k] + B > n_rows || !(lr[k] > 0.0f)) {
            set_error("st_mlp_train: step %d: rows [%lld, %lld) outside the %lld rows, or lr <= 0", k,
                      (long long)row_start[k], (long long)(row_start[k] + B), (long long)n_rows);
            return ST_EINVAL;
        }
    if (steps == 0) return ST_OK;
    double* d_loss = nullptr;
    if (loss_out) {
        cudaError_t e = cudaMallocAsync((void**)&d_loss, (size_t)steps * sizeof(double), n->stream);
        if (e != cudaSuccess) return cuda_fail(e, "st_mlp_train: loss buffer");
    }
    // the first step eagerly (it also sets the kernels' attributes and fills the
    // tensor-map cache before the capture), the rest replayed from a graph
    int rc = st_mlp_loss_grad_residual(n, x_rows + row_start[0] * MLP_IN, r_rows + row_start[0] * MLP_OUT, B, nullptr,
                                       nullptr);
    if (rc == ST_OK && d_loss) {
        cudaError_t e = cudaMemcpyAsync(d_loss, n->loss, sizeof(double), cudaMemcpyDeviceToDevice, n->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: loss copy");
    }
    if (rc == ST_OK) rc = st_mlp_adam_step(n, lr[0], beta1, beta2, eps);
    if (rc == ST_OK && steps > 1)
        rc = train_replayed(n, x_rows, r_rows, B, steps, row_start, lr, beta1, beta2, eps, d_loss);
    if (d_loss) {
        if (rc == ST_OK) {
            cudaError_t e = cudaMemcpyAsync(loss_out, d_loss, (size_t)steps * sizeof(double), cudaMemcpyDeviceToHost,
                                            n->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "st_mlp_train: loss download");
        }
        cudaFreeAsync(d_loss, n->stream);
    }
    if (rc) return rc;
    return check_status(n, "st_mlp_train");
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
    if (n_turns < 0 || ctx->n > n->max_batch) {
        set_error("st_track_surrogate: need n_turns >= 0 and n_particles <= the network's max_batch");
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
        mlp_pack_state<<<(Bp + 127) / 128, 128, 0, n->stream>>>(ctx->xpx, ctx->ypy, ctx->tpt, B, Bp, n->head, n->X0);
        rc = mlp_forward_layers(n, Bp, false);
        if (rc) break;
        surrogate_apply<<<(B + 127) / 128, 128, 0, n->stream>>>(n->Y, B, n->head, ctx->xpx, ctx->ypy, ctx->tpt,
                                                                ctx->sxy, ctx->sz, ctx->lost, spin_sum);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "st_track_surrogate: spin step");
            break;
        }
        rc = ctx->precision == ST_MIXED ? launch_track_mixed_orbit(ctx, 1) : launch_track_orbit(ctx, 1);
    }
    n->stream = keep;
    return rc;
}

}  // extern "C"
