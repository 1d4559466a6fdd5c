// FP64 tracker kernel over one particle ensemble (persistent warp ranges,
// equal FP64 work per SM), its launcher and the state pack/unpack kernels.
// The per-particle integrators are fp64_track_particle in track_fp64.cuh
// (Romberg orders) and fp64_track_particle_mid in track_mid.cuh (midpoint
// schemes).
#include <cstdio>

#include "track_mid.cuh"

namespace st {

// 2 blocks of 128 per SM (up to 255 registers, no spills): the FP64 pipe is
// saturated from 4 resident warps per SM, and the larger register budget
// schedules the dependency chains better than 3 blocks with 168 registers
// (measured 1.6% faster on the RHIC-like ring).
template <int K, bool SPIN = true, bool EXT = false>
__global__ void __launch_bounds__(128, 2) track_fp64_kernel(const void* __restrict__ blob, uint32_t blob_bytes,
                                                         uint32_t seq_offset, int n_seq, RefConst ref,
                                                         double2* __restrict__ xpx, double2* __restrict__ ypy,
                                                         double2* __restrict__ tpt, double2* __restrict__ sxy,
                                                         double* __restrict__ szp, uint8_t* __restrict__ lost,
                                                         int n, int n_turns, int32_t* __restrict__ status,
                                                         TurnOut tq) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ double qcache[(2 * QC_N + 2) * 128];
    if (!stage_to_smem(smem, blob, blob_bytes, &bar, status)) return;
    const DevElem* table = (const DevElem*)smem;
    const uint16_t* seq = (const uint16_t*)(smem + seq_offset);

    // Every block owns a contiguous, equal share of whole warps of particles;
    // the grid is (#SMs x resident blocks per SM), so every SM gets the same
    // amount of FP64 work.
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t n_warps = ((int64_t)n + 31) / 32;
    const int64_t w_begin = (int64_t)blockIdx.x * n_warps / gridDim.x;
    const int64_t w_end = (int64_t)(blockIdx.x + 1) * n_warps / gridDim.x;
    for (int64_t wi = w_begin + (threadIdx.x >> 5); wi < w_end; wi += wpb) {
    const int64_t i = wi * 32 + lane;
    if (i >= n || lost[i]) continue;

    if constexpr (K < 0)   // midpoint schemes: K = ST_SPIN_MID_HALF or ST_SPIN_MID_KICK
        fp64_track_particle_mid<K == ST_SPIN_MID_KICK>(table, seq, n_seq, ref, xpx, ypy, tpt, sxy, szp, lost, i,
                                                        n_turns, qcache, tq, status);
    else
        fp64_track_particle<K, SPIN, EXT>(table, seq, n_seq, ref, xpx, ypy, tpt, sxy, szp, lost, i, n_turns,
                                          qcache, tq, status);
    }  // particle loop
}

__global__ void pack_kernel(const double* __restrict__ z, const double* __restrict__ s, double2* xpx, double2* ypy,
                            double2* tpt, double2* sxy, double* sz, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    xpx[i] = make_double2(z[i], z[n + i]);
    ypy[i] = make_double2(z[2 * n + i], z[3 * n + i]);
    tpt[i] = make_double2(z[4 * n + i], z[5 * n + i]);
    sxy[i] = make_double2(s[i], s[n + i]);
    sz[i] = s[2 * n + i];
}

__global__ void unpack_kernel(double* __restrict__ z, double* __restrict__ s, const double2* xpx, const double2* ypy,
                              const double2* tpt, const double2* sxy, const double* sz, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = xpx[i], b = ypy[i], c = tpt[i], d = sxy[i];
    z[i] = a.x;
    z[n + i] = a.y;
    z[2 * n + i] = b.x;
    z[3 * n + i] = b.y;
    z[4 * n + i] = c.x;
    z[5 * n + i] = c.y;
    s[i] = d.x;
    s[n + i] = d.y;
    s[2 * n + i] = sz[i];
}

int launch_pack(st_ctx* ctx, const double* z, const double* s) {
    int64_t n = ctx->n;
    int threads = 256;
    unsigned blocks = (unsigned)((n + threads - 1) / threads);
    pack_kernel<<<blocks, threads, 0, ctx->stream>>>(z, s, ctx->xpx, ctx->ypy, ctx->tpt, ctx->sxy, ctx->sz, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "pack kernel launch");
}

int launch_unpack(st_ctx* ctx, double* z, double* s) {
    int64_t n = ctx->n;
    int threads = 256;
    unsigned blocks = (unsigned)((n + threads - 1) / threads);
    unpack_kernel<<<blocks, threads, 0, ctx->stream>>>(z, s, ctx->xpx, ctx->ypy, ctx->tpt, ctx->sxy, ctx->sz, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ST_OK : cuda_fail(e, "unpack kernel launch");
}

template <int K, bool SPIN, bool EXT>
static int launch_k_(st_ctx* ctx, int n_turns, const TurnOut& tq) {
    const LatticeImpl& L = ctx->lat->impl;
    const int threads = ctx->block_threads;
    const size_t smem = L.blob_bytes;
    static PerDeviceOnce attr_set;
    int rc0 = once_per_device(
        attr_set,
        [] {
            return cudaFuncSetAttribute(track_fp64_kernel<K, SPIN, EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024);
        },
        "cudaFuncSetAttribute(fp64 tracker)");
    if (rc0) return rc0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_fp64_kernel<K, SPIN, EXT>, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 tracker occupancy query");
    if (per_sm < 1) {
        set_error("fp64 tracker: block of %d threads with %zu B shared memory does not fit on an SM", threads,
                  smem);
        return ST_EINVAL;
    }
    // never more blocks than warps of particles
    const int64_t n_warps = (ctx->n + 31) / 32;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_warps) grid = n_warps;
    const int tpl = ctx->turns_per_launch;
    for (int t = 0; t < n_turns; t += tpl) {
        int nt = n_turns - t < tpl ? n_turns - t : tpl;
        track_fp64_kernel<K, SPIN, EXT><<<(unsigned)grid, threads, smem, ctx->stream>>>(
            L.d_blob, (uint32_t)L.blob_bytes, (uint32_t)L.seq_offset, L.n_elements, L.ref, ctx->xpx, ctx->ypy,
            ctx->tpt, ctx->sxy, ctx->sz, ctx->lost, (int)ctx->n, nt, ctx->status, tq);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "fp64 tracker launch");
    }
    return ST_OK;
}

// The extended instantiation only for lattices with extended elements; the
// midpoint schemes have one instantiation each, with every element type.
template <int K, bool SPIN = true>
static int launch_k(st_ctx* ctx, int n_turns, const TurnOut& tq) {
    if constexpr (K < 0)
        return launch_k_<K, true, true>(ctx, n_turns, tq);
    else
        return ctx->lat->impl.has_ext ? launch_k_<K, SPIN, true>(ctx, n_turns, tq)
                                         : launch_k_<K, SPIN, false>(ctx, n_turns, tq);
}

// Orbit only (spins untouched): the orbit maps of the FP64 tracker without the
// precession, level products and spin rotation.
int launch_track_orbit(st_ctx* ctx, int n_turns) {
    if (ctx->lat->impl.blob_bytes > 200 * 1024) {
        set_error("lattice table of %zu bytes exceeds the 200 KiB shared-memory budget",
                  ctx->lat->impl.blob_bytes);
        return ST_EINVAL;
    }
    if (ctx->block_threads > 128) {
        set_error("orbit tracker: block_threads must be <= 128");
        return ST_EINVAL;
    }
    return launch_k<0, false>(ctx, n_turns, TurnOut{nullptr, nullptr, 0, {}});
}

int launch_track_fp64(st_ctx* ctx, int n_turns, int spin_order, const TurnOut& out) {
    if (ctx->lat->impl.blob_bytes > 200 * 1024) {
        set_error("lattice table of %zu bytes exceeds the 200 KiB shared-memory budget",
                  ctx->lat->impl.blob_bytes);
        return ST_EINVAL;
    }
    if (ctx->block_threads > 128) {
        set_error("fp64 tracker: block_threads must be <= 128");
        return ST_EINVAL;
    }
    switch (spin_order) {
    case ST_SPIN_MID_HALF: return launch_k<ST_SPIN_MID_HALF>(ctx, n_turns, out);
    case ST_SPIN_MID_KICK: return launch_k<ST_SPIN_MID_KICK>(ctx, n_turns, out);
    case 0: return launch_k<0>(ctx, n_turns, out);
    case 1: return launch_k<1>(ctx, n_turns, out);
    case 2: return launch_k<2>(ctx, n_turns, out);
    case 3: return launch_k<3>(ctx, n_turns, out);
    case 4: return launch_k<4>(ctx, n_turns, out);
    }
    set_error("spin_order out of range");
    return ST_EINVAL;
}

int launch_track_fp64(st_ctx* ctx, int n_turns, int spin_order) {
    return launch_track_fp64(ctx, n_turns, spin_order, TurnOut{nullptr, nullptr, 0, {}});
}

// One turn, storing every particle's one-turn quaternion (sign-aligned with q_ref).
int launch_track_turn_map(st_ctx* ctx, int spin_order, double* q_out, const double* q_ref) {
    TurnOut out{q_out, nullptr, ctx->n, {q_ref[0], q_ref[1], q_ref[2], q_ref[3]}};
    return launch_track_fp64(ctx, 1, spin_order, out);
}

// n_turns with the spin at the start of the lattice summed after every turn.
int launch_track_average(st_ctx* ctx, int n_turns, int spin_order, double* spin_sum) {
    TurnOut out{nullptr, spin_sum, ctx->n, {1.0, 0.0, 0.0, 0.0}};
    return launch_track_fp64(ctx, n_turns, spin_order, out);
}

}  // namespace st
