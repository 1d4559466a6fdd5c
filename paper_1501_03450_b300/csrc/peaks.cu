// Arithmetic-throughput probes: sustained FP64 and FP32 fused multiply-add
// rates of the current device, measured with independent FMA chains and CUDA
// events.  The tracker's roofline denominators come from here.
#include "st_internal.cuh"
#include "device_common.cuh"

namespace st {

template <typename T>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-12345.0) out[0] = s;   // keeps the chains alive, never taken
}

template <typename T>
static int probe(int blocks_per_sm, int iters, double* fma_per_s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "probe: device query");
    T* out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&out, sizeof(T));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int threads = 256;
    const int blocks = sms * blocks_per_sm;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0);
        fma_probe_kernel<T><<<blocks, threads>>>(out, iters, (T)0.9999999, (T)1e-7);
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best_ms) best_ms = ms;   // first run is warm-up
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "probe kernel");
    double n_fma = (double)blocks * threads * 8.0 * iters;
    *fma_per_s = n_fma / (best_ms * 1e-3);
    return ST_OK;
}

// Packed FP32x2 chains (FFMA2: two fused multiply-adds per instruction).
__global__ void ffma2_probe_kernel(float* out, int iters, float a, float b) {
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    float2 x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = make_float2((float)threadIdx.x * 1e-3f + (float)j, (float)j + 0.5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
    if (s == -12345.0f) out[0] = s;   // keeps the chains alive, never taken
}

static int probe_ffma2(int blocks_per_sm, int iters, double* fma_per_s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "probe: device query");
    float* out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&out, sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int threads = 256;
    const int blocks = sms * blocks_per_sm;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0);
        ffma2_probe_kernel<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best_ms) best_ms = ms;   // first run is warm-up
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "FFMA2 probe kernel");
    *fma_per_s = (double)blocks * threads * 16.0 * iters / (best_ms * 1e-3);
    return ST_OK;
}

}  // namespace st

extern "C" int st_measure_fp32x2_peak(double* fp32_flops) {
    if (!fp32_flops) {
        st::set_error("st_measure_fp32x2_peak: null pointer");
        return ST_EINVAL;
    }
    double r = 0;
    int rc = st::probe_ffma2(8, 100000, &r);
    if (rc) return rc;
    *fp32_flops = 2.0 * r;
    return ST_OK;
}

extern "C" int st_measure_peaks(double* fp64_flops, double* fp32_flops) {
    if (!fp64_flops || !fp32_flops) {
        st::set_error("st_measure_peaks: null pointer");
        return ST_EINVAL;
    }
    double r64 = 0, r32 = 0;
    int rc = st::probe<double>(4, 20000, &r64);
    if (rc) return rc;
    rc = st::probe<float>(8, 200000, &r32);
    if (rc) return rc;
    *fp64_flops = 2.0 * r64;
    *fp32_flops = 2.0 * r32;
    return ST_OK;
}

// ---- bounded-wait self-test ------------------------------------------------
namespace st {

// One block: thread 0 initialises an mbarrier that expects one arrival which
// nothing ever makes (no copy is issued), every thread then runs the
// library's bounded wait on it; the wait gives up after limit_ns, and thread
// 0 records the outcome and the elapsed time.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int32_t* status, unsigned long long* elapsed_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t t0 = global_timer_ns();
    const bool ok = mbar_wait_bounded(&bar, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) {
        *status = ok ? STATUS_OK : STATUS_TMA_TIMEOUT;
        *elapsed_ns = global_timer_ns() - t0;
    }
}

}  // namespace st

extern "C" int st_selftest_bounded_wait(double limit_s, double* elapsed_s) {
    if (!elapsed_s || !(limit_s >= 1e-4) || !(limit_s <= 2.0)) {
        st::set_error("st_selftest_bounded_wait: need elapsed_s and 1e-4 <= limit_s <= 2");
        return ST_EINVAL;
    }
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 16);
    if (e != cudaSuccess) return st::cuda_fail(e, "st_selftest_bounded_wait: allocation");
    int32_t* d_status = (int32_t*)buf;
    unsigned long long* d_elapsed = (unsigned long long*)((char*)buf + 8);
    st::bounded_wait_selftest_kernel<<<1, 32>>>((uint64_t)(limit_s * 1e9), d_status, d_elapsed);
    e = cudaGetLastError();
    int32_t h_status = -1;
    unsigned long long h_elapsed = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h_status, d_status, sizeof(h_status), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h_elapsed, d_elapsed, sizeof(h_elapsed), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return st::cuda_fail(e, "st_selftest_bounded_wait");
    *elapsed_s = (double)h_elapsed * 1e-9;
    if (h_status != st::STATUS_OK) {
        st::set_error("st_selftest_bounded_wait: the wait gave up after %.3g s (status %d)", *elapsed_s, h_status);
        return ST_ETIMEOUT;
    }
    return ST_OK;
}
