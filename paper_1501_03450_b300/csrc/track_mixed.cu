// Mixed-precision tracker kernel over one particle ensemble and its
// launcher; the per-particle integrator is mixed_track_particle in
// track_mixed.cuh.
#include "track_mixed_mid.cuh"

namespace st {

// 2 blocks of 128 per SM (up to 255 registers): 13% faster than 3 blocks with a
// 168-register cap on the RHIC-like ring (fewer warps, but no rematerialisation).
template <int K, bool SPIN = true, bool FR = false, bool EXT = false, bool O4 = false, bool RB = false>
__global__ void __launch_bounds__(128, 2) track_mixed_kernel(const void* __restrict__ blob, uint32_t blob_bytes,
                                                            uint32_t seq_offset, uint32_t rho_offset, int n_seq,
                                                            RefConst ref, double2* __restrict__ xpx,
                                                            double2* __restrict__ ypy, double2* __restrict__ tpt,
                                                            double2* __restrict__ sxy, double* __restrict__ szp,
                                                            uint8_t* __restrict__ lost, int n, int n_turns,
                                                            int32_t* __restrict__ status,
                                                            double* __restrict__ spin_sum) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    if (!stage_to_smem(smem, blob, blob_bytes, &bar, status)) return;
    const MixElem* table = (const MixElem*)smem;
    const uint16_t* seq = (const uint16_t*)(smem + seq_offset);
    const float2* rho = (const float2*)(smem + rho_offset);

    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t n_warps = ((int64_t)n + 31) / 32;
    const int64_t w_begin = (int64_t)blockIdx.x * n_warps / gridDim.x;
    const int64_t w_end = (int64_t)(blockIdx.x + 1) * n_warps / gridDim.x;
    for (int64_t wi = w_begin + (threadIdx.x >> 5); wi < w_end; wi += wpb) {
        const int64_t i = wi * 32 + lane;
        if (i >= n || lost[i]) continue;

        mixed_track_particle<K, SPIN, FR, EXT, O4, RB>(table, seq, rho, n_seq, ref, xpx, ypy, tpt, sxy, szp, lost,
                                                       i, n_turns, status, spin_sum, n);
    }
}

// The midpoint spin schemes (KICK: split-kick placement), a separate kernel.
template <bool KICK, bool FR, bool EXT, bool RB = false>
__global__ void __launch_bounds__(128, 2) track_mixed_mid_kernel(const void* __restrict__ blob, uint32_t blob_bytes,
                                                                uint32_t seq_offset, uint32_t rho_offset, int n_seq,
                                                                RefConst ref, double2* __restrict__ xpx,
                                                                double2* __restrict__ ypy, double2* __restrict__ tpt,
                                                                double2* __restrict__ sxy, double* __restrict__ szp,
                                                                uint8_t* __restrict__ lost, int n, int n_turns,
                                                                int32_t* __restrict__ status,
                                                                double* __restrict__ spin_sum) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    if (!stage_to_smem(smem, blob, blob_bytes, &bar, status)) return;
    const MixElem* table = (const MixElem*)smem;
    const uint16_t* seq = (const uint16_t*)(smem + seq_offset);
    const float2* rho = (const float2*)(smem + rho_offset);
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t n_warps = ((int64_t)n + 31) / 32;
    const int64_t w_begin = (int64_t)blockIdx.x * n_warps / gridDim.x;
    const int64_t w_end = (int64_t)(blockIdx.x + 1) * n_warps / gridDim.x;
    for (int64_t wi = w_begin + (threadIdx.x >> 5); wi < w_end; wi += wpb) {
        const int64_t i = wi * 32 + lane;
        if (i >= n || lost[i]) continue;
        mixed_track_particle_mid<KICK, FR, EXT, RB>(table, seq, rho, n_seq, ref, xpx, ypy, tpt, sxy, szp, lost, i,
                                                    n_turns, status, spin_sum, n);
    }
}

template <bool KICK, bool FR, bool EXT, bool RB = false>
static int launch_mixed_mid_(st_ctx* ctx, int n_turns, double* spin_sum) {
    const LatticeImpl& L = ctx->lat->impl;
    const int threads = ctx->block_threads;
    const size_t smem = L.mix_bytes;
    static PerDeviceOnce attr_set;
    int rc0 = once_per_device(
        attr_set,
        [] {
            return cudaFuncSetAttribute(track_mixed_mid_kernel<KICK, FR, EXT, RB>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        },
        "cudaFuncSetAttribute(mixed midpoint tracker)");
    if (rc0) return rc0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_mixed_mid_kernel<KICK, FR, EXT, RB>, threads,
                                                          smem);
    if (e != cudaSuccess) return cuda_fail(e, "mixed midpoint tracker occupancy query");
    if (per_sm < 1) {
        set_error("mixed midpoint tracker: block of %d threads with %zu B shared memory does not fit on an SM",
                  threads, smem);
        return ST_EINVAL;
    }
    const int64_t n_warps = (ctx->n + 31) / 32;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_warps) grid = n_warps;
    const int tpl = ctx->turns_per_launch;
    for (int t = 0; t < n_turns; t += tpl) {
        int nt = n_turns - t < tpl ? n_turns - t : tpl;
        track_mixed_mid_kernel<KICK, FR, EXT, RB><<<(unsigned)grid, threads, smem, ctx->stream>>>(
            L.d_mix, (uint32_t)L.mix_bytes, (uint32_t)L.mix_seq_offset, (uint32_t)L.mix_rho_offset, L.n_elements,
            L.ref, ctx->xpx, ctx->ypy, ctx->tpt, ctx->sxy, ctx->sz, ctx->lost, (int)ctx->n, nt, ctx->status,
            spin_sum);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "mixed midpoint tracker launch");
    }
    return ST_OK;
}

// Lattices with TEAPOT bends run the extended instantiation (which also
// decodes fringe-kick entries), the others the one their fringe kicks need.
template <bool KICK>
static int launch_mixed_mid(st_ctx* ctx, int n_turns, double* spin_sum) {
    const LatticeImpl& L = ctx->lat->impl;
    if (L.mix_rb) return launch_mixed_mid_<KICK, true, true, true>(ctx, n_turns, spin_sum);
    if (L.mix_ext) return launch_mixed_mid_<KICK, true, true>(ctx, n_turns, spin_sum);
    return L.mix_fringe ? launch_mixed_mid_<KICK, true, false>(ctx, n_turns, spin_sum)
                        : launch_mixed_mid_<KICK, false, false>(ctx, n_turns, spin_sum);
}

template <int K, bool SPIN, bool FR, bool EXT, bool O4 = false, bool RB = false>
static int launch_mixed_k_(st_ctx* ctx, int n_turns, double* spin_sum) {
    const LatticeImpl& L = ctx->lat->impl;
    const int threads = ctx->block_threads;
    const size_t smem = L.mix_bytes;
    static PerDeviceOnce attr_set;
    int rc0 = once_per_device(
        attr_set,
        [] {
            return cudaFuncSetAttribute(track_mixed_kernel<K, SPIN, FR, EXT, O4, RB>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        },
        "cudaFuncSetAttribute(mixed tracker)");
    if (rc0) return rc0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_mixed_kernel<K, SPIN, FR, EXT, O4, RB>, threads,
                                                          smem);
    if (e != cudaSuccess) return cuda_fail(e, "mixed tracker occupancy query");
    if (per_sm < 1) {
        set_error("mixed tracker: block of %d threads with %zu B shared memory does not fit on an SM", threads, smem);
        return ST_EINVAL;
    }
    const int64_t n_warps = (ctx->n + 31) / 32;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_warps) grid = n_warps;
    const int tpl = ctx->turns_per_launch;
    for (int t = 0; t < n_turns; t += tpl) {
        int nt = n_turns - t < tpl ? n_turns - t : tpl;
        track_mixed_kernel<K, SPIN, FR, EXT, O4, RB><<<(unsigned)grid, threads, smem, ctx->stream>>>(
            L.d_mix, (uint32_t)L.mix_bytes, (uint32_t)L.mix_seq_offset, (uint32_t)L.mix_rho_offset, L.n_elements,
            L.ref, ctx->xpx, ctx->ypy, ctx->tpt, ctx->sxy, ctx->sz, ctx->lost, (int)ctx->n, nt, ctx->status,
            spin_sum);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "mixed tracker launch");
    }
    return ST_OK;
}

// The instantiation that decodes fringe-kick entries only for lattices with
// them; lattices with TEAPOT bends or solenoids run the extended one (fringe
// entries too), lattices with fourth-order slices the extended one with those,
// lattices with rectangular bends the one with everything.
template <int K, bool SPIN = true>
static int launch_mixed_k(st_ctx* ctx, int n_turns, double* spin_sum = nullptr) {
    const LatticeImpl& L = ctx->lat->impl;
    if (L.mix_rb) return launch_mixed_k_<K, SPIN, true, true, true, true>(ctx, n_turns, spin_sum);
    if (L.mix_o4) return launch_mixed_k_<K, SPIN, true, true, true>(ctx, n_turns, spin_sum);
    if (L.mix_ext) return launch_mixed_k_<K, SPIN, true, true>(ctx, n_turns, spin_sum);
    return L.mix_fringe ? launch_mixed_k_<K, SPIN, true, false>(ctx, n_turns, spin_sum)
                        : launch_mixed_k_<K, SPIN, false, false>(ctx, n_turns, spin_sum);
}

// Orbit only, in the mixed tracker's compensated arithmetic (spins untouched).
int launch_track_mixed_orbit(st_ctx* ctx, int n_turns) {
    if (ctx->lat->impl.mix_bytes > 200 * 1024 || ctx->block_threads > 128) {
        set_error("mixed orbit tracker: lattice table too large or block_threads > 128");
        return ST_EINVAL;
    }
    return launch_mixed_k<0, false>(ctx, n_turns);
}

int launch_track_mixed(st_ctx* ctx, int n_turns, int spin_order, double* spin_sum) {
    const LatticeImpl& L = ctx->lat->impl;
    if (!L.d_mix) {
        set_error("mixed tracker: lattice has no mixed-precision tables");
        return ST_ESTATE;
    }
    if (L.mix_bytes > 200 * 1024) {
        set_error("mixed-precision tables of %zu bytes exceed the 200 KiB shared-memory budget", L.mix_bytes);
        return ST_EINVAL;
    }
    if (ctx->block_threads > 128) {
        set_error("mixed tracker: block_threads must be <= 128");
        return ST_EINVAL;
    }
    switch (spin_order) {
    case ST_SPIN_MID_HALF: return launch_mixed_mid<false>(ctx, n_turns, spin_sum);
    case ST_SPIN_MID_KICK: return launch_mixed_mid<true>(ctx, n_turns, spin_sum);
    case 0: return launch_mixed_k<0>(ctx, n_turns, spin_sum);
    case 1: return launch_mixed_k<1>(ctx, n_turns, spin_sum);
    case 2: return launch_mixed_k<2>(ctx, n_turns, spin_sum);
    case 3: return launch_mixed_k<3>(ctx, n_turns, spin_sum);
    case 4: return launch_mixed_k<4>(ctx, n_turns, spin_sum);
    }
    set_error("spin_order out of range");
    return ST_EINVAL;
}

}  // namespace st
