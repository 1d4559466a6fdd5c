// Device helpers shared by the tracking kernels: bulk copy of the lattice into
// shared memory through the TMA engine (cp.async.bulk + mbarrier, bounded
// wait), and small quaternion routines in FP64.
#pragma once

#include "st_internal.cuh"

namespace st {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared, completion signalled on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (about `limit_ns` of wall time) for the phase with the given
// parity of `bar` to complete.
__device__ __forceinline__ bool mbar_wait_bounded_parity(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint64_t limit_ns) {
    return mbar_wait_bounded_parity(bar, 0, limit_ns);
}

// Issue the bulk copies of `bytes` (multiple of 16) into shared memory on an
// already initialised barrier (one thread calls this).
__device__ __forceinline__ void issue_bulk_stage(void* smem, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, bytes);
    const char* s = (const char*)gsrc;
    char* d = (char*)smem;
    uint32_t off = 0;
    while (off < bytes) {
        uint32_t c = bytes - off < 65536u ? bytes - off : 65536u;
        bulk_copy_g2s(d + off, s + off, c, bar);
        off += c;
    }
}

// Stage `bytes` (multiple of 16) of the lattice blob into shared memory.  All
// threads of the block call this; returns false (and sets *status) if the
// copy did not complete within about one second.
__device__ __forceinline__ bool stage_to_smem(void* smem, const void* gsrc, uint32_t bytes, uint64_t* bar,
                                              int32_t* status) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, bytes);
        // chunks of at most 64 KiB keep each copy well inside the transaction-count range
        const char* s = (const char*)gsrc;
        char* d = (char*)smem;
        uint32_t off = 0;
        while (off < bytes) {
            uint32_t c = bytes - off < 65536u ? bytes - off : 65536u;
            bulk_copy_g2s(d + off, s + off, c, bar);
            off += c;
        }
    }
    bool ok = mbar_wait_bounded(bar, 1000000000ull);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(status, STATUS_TMA_TIMEOUT);
        // give the copy in flight one more bounded chance to land before the
        // block exits
        mbar_wait_bounded(bar, 1000000000ull);
    }
    __syncthreads();
    return ok;
}

// ---- quaternions (scalar first), FP64 ----------------------------------
struct Quat {
    double w, x, y, z;
};

__device__ __forceinline__ Quat qmul(const Quat& a, const Quat& b) {
    Quat o;
    o.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
    o.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
    o.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
    o.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
    return o;
}

// Square of a unit quaternion: (w^2 - |v|^2, 2 w v) with w^2 - |v|^2 = 2 w^2 - 1
// for |q| = 1 (one fused operation instead of four products).
__device__ __forceinline__ Quat qsquare(const Quat& a) {
    const double w2 = a.w + a.w;
    return Quat{fma(w2, a.w, -1.0), w2 * a.x, w2 * a.y, w2 * a.z};
}

__device__ __forceinline__ Quat qnormalize(const Quat& a) {
    double r = rsqrt(a.w * a.w + a.x * a.x + a.y * a.y + a.z * a.z);
    return Quat{a.w * r, a.x * r, a.y * r, a.z * r};
}

// Unit quaternion of the rotation by |w| about w^, with library sincos.
__device__ __forceinline__ Quat quat_from_rotvec_lib(double wx, double wy, double wz) {
    double th2 = wx * wx + wy * wy + wz * wz;
    if (th2 > 0.0) {
        double r = rsqrt(th2);
        double th = th2 * r;
        double s, c;
        sincos(0.5 * th, &s, &c);
        double f = s * r;
        return Quat{c, f * wx, f * wy, f * wz};
    }
    return Quat{1.0, 0.0, 0.0, 0.0};
}

// Taylor coefficients of cos(t/2) and sin(t/2)/t as power series in u = t^2:
//   cos(t/2)   = sum_n (-1)^n u^n / (4^n (2n)!)
//   sin(t/2)/t = sum_n (-1)^n u^n / (2 4^n (2n+1)!)
// (exact rationals, fixed at compile time by template recursion).
template <int N> struct Fact { static constexpr double v = (double)N * Fact<N - 1>::v; };
template <> struct Fact<0> { static constexpr double v = 1.0; };
template <int N> struct Pow4 { static constexpr double v = 4.0 * Pow4<N - 1>::v; };
template <> struct Pow4<0> { static constexpr double v = 1.0; };
template <int N> struct HalfCosCoef {
    static constexpr double v = (N % 2 ? -1.0 : 1.0) / (Pow4<N>::v * Fact<2 * N>::v);
};
template <int N> struct HalfSincCoef {
    static constexpr double v = (N % 2 ? -1.0 : 1.0) / (2.0 * Pow4<N>::v * Fact<2 * N + 1>::v);
};

template <int N>
struct HalfAngleHorner {   // continues Horner's rule from degree N down to 0
    static __device__ __forceinline__ void step(double u, double& c, double& f) {
        c = fma(c, u, HalfCosCoef<N>::v);
        f = fma(f, u, HalfSincCoef<N>::v);
        HalfAngleHorner<N - 1>::step(u, c, f);
    }
};
template <>
struct HalfAngleHorner<-1> {
    static __device__ __forceinline__ void step(double, double&, double&) {}
};

template <int DEG>
__device__ __forceinline__ void half_angle_series(double u, double& c, double& f) {
    c = HalfCosCoef<DEG>::v;
    f = HalfSincCoef<DEG>::v;
    HalfAngleHorner<DEG - 1>::step(u, c, f);
}

// High words of the series thresholds 4e-6, 4e-4 and 0.04: for a non-negative
// double the high 32 bits, read as a signed integer, order it like its value,
// so the thresholds are tested on the integer pipe (the FP64 pipe is the
// tracker's bottleneck).  Each comparison is conservative by < 1e-6 relative.
constexpr int HIWORD_4EM6 = 0x3ed0c6f7;
constexpr int HIWORD_4EM4 = 0x3f3a36e2;
constexpr int HIWORD_0P04 = 0x3fa47ae1;

// Unit quaternion of the rotation by |w| about w^ without library calls:
// q = (cos(t/2), sin(t/2)/t * w) with t^2 = w.w, both even functions of t
// evaluated as truncated Taylor series in u = t^2: degree 2 for u < 4e-6,
// 3 for u < 4e-4, 5 for u < 0.04, 11 for u <= 4 (truncation below 3e-21
// relative in every range).  Larger angles are halved until u <= 4 and the
// quaternion squared back.  The degree is the largest one any active lane of
// the warp needs, so that the branch stays uniform (a lane never gets less
// than its own u requires).
__device__ __forceinline__ Quat quat_from_rotvec(double wx, double wy, double wz) {
    double u = wx * wx + wy * wy + wz * wz;
    double c, f;
    const int hu = __double2hiint(u);   // NaN orders above every threshold
    int need = hu < HIWORD_4EM6 ? 2 : hu < HIWORD_4EM4 ? 3 : hu < HIWORD_0P04 ? 5 : 11;
    need = __reduce_max_sync(__activemask(), need);
    if (need <= 5) {
        if (need == 2) half_angle_series<2>(u, c, f);
        else if (need == 3) half_angle_series<3>(u, c, f);
        else half_angle_series<5>(u, c, f);
        return Quat{c, f * wx, f * wy, f * wz};
    }
    int m = 0;
    double scale = 1.0;
    while (u > 4.0 && m < 60) {
        u *= 0.25;
        scale *= 0.5;
        ++m;
    }
    half_angle_series<11>(u, c, f);
    f *= scale;
    Quat q{c, f * wx, f * wy, f * wz};
    for (int k = 0; k < m; ++k) q = qsquare(q);
    return q;
}

// S <- Q S conj(Q) for a unit quaternion Q.
__device__ __forceinline__ void rotate_vec(const Quat& q, double& sx, double& sy, double& sz) {
    // t = 2 v x S ; S' = S + w t + v x t
    double tx = 2.0 * (q.y * sz - q.z * sy);
    double ty = 2.0 * (q.z * sx - q.x * sz);
    double tz = 2.0 * (q.x * sy - q.y * sx);
    double nx = sx + q.w * tx + (q.y * tz - q.z * ty);
    double ny = sy + q.w * ty + (q.z * tx - q.x * tz);
    double nz = sz + q.w * tz + (q.x * ty - q.y * tx);
    sx = nx;
    sy = ny;
    sz = nz;
}

}  // namespace st
