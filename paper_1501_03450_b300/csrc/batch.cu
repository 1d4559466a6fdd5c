// Batched tracking of many independent jobs (rings of uneven length, particle
// counts and energies) in one persistent launch.
//
// Work is cut into items of one block's worth of particles of one job and
// ordered by estimated cost, largest first.  A persistent grid (#SMs x
// resident blocks) pops items from a device work queue (one atomic counter,
// reset before every launch); for each item the block stages that job's
// lattice into shared memory with a bulk TMA copy (mbarrier, phase-tracked,
// bounded wait) and every thread tracks one particle with the same
// per-particle integrator as the single-job kernels, so results are
// identical to tracking each job on its own.  The turn loop (queue reset +
// kernel per chunk of turns) is captured once into a CUDA graph and replayed.
// An autotuner times block size, turns per launch and the register budget
// (two launch-bound variants) on the live state, restoring it after every
// trial.
#include <algorithm>
#include <cstring>
#include <vector>

#include "track_mid.cuh"
#include "track_mixed_mid.cuh"

namespace st {

struct JobDesc {
    const void* blob;
    uint32_t blob_bytes;
    uint32_t seq_offset;
    uint32_t rho_offset;
    int32_t n_seq;
    RefConst ref;
    double2 *xpx, *ypy, *tpt, *sxy;
    double* sz;
    uint8_t* lost;
    int64_t n;
};

struct WorkItem {
    int32_t job;
    int32_t first;
    int32_t count;
    int32_t pad_;
};

// Pop items until the queue is empty.  Returns false if a lattice staging
// wait expired (status set).
template <class Body>
__device__ __forceinline__ void batch_loop(const JobDesc* __restrict__ jobs, const WorkItem* __restrict__ items,
                                           int n_items, int32_t* queue, int32_t* status, unsigned char* smem,
                                           uint64_t* bar, Body body) {
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int cur_job = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        if constexpr (kChecked) {
            if (w.job < 0 || w.first < 0 || w.count < 0 || w.count > (int)blockDim.x) {
                if (threadIdx.x == 0) atomicExch(status, STATUS_BOUNDS);
                __syncthreads();
                continue;
            }
        }
        const JobDesc J = jobs[w.job];
        if constexpr (kChecked) {
            if ((int64_t)w.first + w.count > J.n) {
                if (threadIdx.x == 0) atomicExch(status, STATUS_BOUNDS);
                __syncthreads();
                continue;
            }
        }
        if (w.job != cur_job) {
            if (threadIdx.x == 0) issue_bulk_stage(smem, J.blob, J.blob_bytes, bar);
            const bool ok = mbar_wait_bounded_parity(bar, phase, 1000000000ull);
            if (!ok) {
                if (threadIdx.x == 0) atomicExch(status, STATUS_TMA_TIMEOUT);
                mbar_wait_bounded_parity(bar, phase, 1000000000ull);
                return;
            }
            phase ^= 1u;
            cur_job = w.job;
        }
        if ((int)threadIdx.x < w.count) {
            const int64_t i = (int64_t)w.first + threadIdx.x;
            if (!J.lost[i]) body(J, i);
        }
        __syncthreads();   // everyone is done with the table and s_item
    }
}

template <int K, int MINB, bool EXT>
__global__ void __launch_bounds__(128, EXT ? (MINB > 2 ? MINB - 1 : MINB) : MINB) track_batch_fp64_kernel(const JobDesc* __restrict__ jobs,
                                                                      const WorkItem* __restrict__ items,
                                                                      int n_items, int32_t* queue, int n_turns,
                                                                      int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ double qcache[(2 * QC_N + 2) * 128];
    batch_loop(jobs, items, n_items, queue, status, smem, &bar, [&](const JobDesc& J, int64_t i) {
        if constexpr (K < 0)   // midpoint schemes
            fp64_track_particle_mid<K == ST_SPIN_MID_KICK>((const DevElem*)smem,
                                                            (const uint16_t*)(smem + J.seq_offset), J.n_seq, J.ref,
                                                            J.xpx, J.ypy, J.tpt, J.sxy, J.sz, J.lost, i, n_turns,
                                                            qcache, TurnOut{nullptr, nullptr, 0, {}}, status);
        else
            fp64_track_particle<K, true, EXT>((const DevElem*)smem, (const uint16_t*)(smem + J.seq_offset), J.n_seq,
                                              J.ref, J.xpx, J.ypy, J.tpt, J.sxy, J.sz, J.lost, i, n_turns, qcache,
                                              TurnOut{nullptr, nullptr, 0, {}}, status);
    });
}

template <int K, int MINB, bool FR = false, bool EXT = false, bool O4 = false, bool RB = false>
__global__ void __launch_bounds__(128, MINB) track_batch_mixed_kernel(const JobDesc* __restrict__ jobs,
                                                                       const WorkItem* __restrict__ items,
                                                                       int n_items, int32_t* queue, int n_turns,
                                                                       int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    batch_loop(jobs, items, n_items, queue, status, smem, &bar, [&](const JobDesc& J, int64_t i) {
        mixed_track_particle<K, true, FR, EXT, O4, RB>((const MixElem*)smem, (const uint16_t*)(smem + J.seq_offset),
                                (const float2*)(smem + J.rho_offset), J.n_seq, J.ref, J.xpx, J.ypy, J.tpt, J.sxy,
                                J.sz, J.lost, i, n_turns, status);
    });
}

// The midpoint spin schemes in mixed precision (KICK: split-kick placement)
template <bool KICK, bool FR = false, bool EXT = false, bool RB = false>
__global__ void __launch_bounds__(128, 2) track_batch_mixed_mid_kernel(const JobDesc* __restrict__ jobs,
                                                                      const WorkItem* __restrict__ items,
                                                                      int n_items, int32_t* queue, int n_turns,
                                                                      int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    batch_loop(jobs, items, n_items, queue, status, smem, &bar, [&](const JobDesc& J, int64_t i) {
        mixed_track_particle_mid<KICK, FR, EXT, RB>((const MixElem*)smem, (const uint16_t*)(smem + J.seq_offset),
                                                    (const float2*)(smem + J.rho_offset), J.n_seq, J.ref, J.xpx,
                                                    J.ypy, J.tpt, J.sxy, J.sz, J.lost, i, n_turns, status, nullptr,
                                                    0);
    });
}

typedef void (*BatchKernel)(const JobDesc*, const WorkItem*, int, int32_t*, int, int32_t*);

template <bool KICK>
static BatchKernel batch_mixed_mid_kernel(bool fr, bool mext, bool mrb) {
    if (mrb) return track_batch_mixed_mid_kernel<KICK, true, true, true>;
    if (mext) return track_batch_mixed_mid_kernel<KICK, true, true>;
    if (fr) return track_batch_mixed_mid_kernel<KICK, true>;
    return track_batch_mixed_mid_kernel<KICK>;
}

// variant 0 / 1 = larger / smaller register budget (fewer / more resident blocks)
// ext: the FP64 instantiation with the extended element set compiled in
// fr: the mixed instantiation that decodes fringe-kick table entries
// mext: the mixed instantiation with TEAPOT bends and solenoids (and fringe
// entries) compiled in, at the larger register budget for both variants;
// mo4: the same with fourth-order slices; mrb: with rectangular bends too
static BatchKernel batch_kernel(int precision, int K, int variant, bool ext, bool fr, bool mext, bool mo4,
                                bool mrb) {
#define ST_SEL(KK)                                                                                            \
    case KK:                                                                                                  \
        if (precision == ST_FP64) {                                                                           \
            if (ext)                                                                                       \
                return variant ? track_batch_fp64_kernel<KK, 3, true> : track_batch_fp64_kernel<KK, 2, true>; \
            return variant ? track_batch_fp64_kernel<KK, 3, false> : track_batch_fp64_kernel<KK, 2, false>;   \
        }                                                                                                     \
        if (mrb) return track_batch_mixed_kernel<KK, 2, true, true, true, true>;                        \
        if (mo4) return track_batch_mixed_kernel<KK, 2, true, true, true>;                              \
        if (mext) return track_batch_mixed_kernel<KK, 2, true, true>;                                   \
        if (fr) return variant ? track_batch_mixed_kernel<KK, 3, true> : track_batch_mixed_kernel<KK, 2, true>; \
        return variant ? track_batch_mixed_kernel<KK, 3> : track_batch_mixed_kernel<KK, 2>;
    switch (K) {
    case ST_SPIN_MID_HALF:
        if (precision != ST_FP64) return batch_mixed_mid_kernel<false>(fr, mext, mrb);
        return variant ? track_batch_fp64_kernel<ST_SPIN_MID_HALF, 3, true>
                       : track_batch_fp64_kernel<ST_SPIN_MID_HALF, 2, true>;
    case ST_SPIN_MID_KICK:
        if (precision != ST_FP64) return batch_mixed_mid_kernel<true>(fr, mext, mrb);
        return variant ? track_batch_fp64_kernel<ST_SPIN_MID_KICK, 3, true>
                       : track_batch_fp64_kernel<ST_SPIN_MID_KICK, 2, true>;
        ST_SEL(0)
        ST_SEL(1)
        ST_SEL(2)
        ST_SEL(3)
        ST_SEL(4)
    }
#undef ST_SEL
    return nullptr;
}

}  // namespace st

using namespace st;

struct st_batch {
    int32_t n_jobs = 0;
    int32_t precision = ST_FP64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool has_ext = false;   // some job's lattice uses fourth-order maps or rectangular bends
    bool mix_fringe = false;   // some job's mixed table has fringe-kick entries
    bool mix_ext = false;      // some job's lattice has TEAPOT bends, solenoids or fourth-order slices
    bool mix_o4 = false;       // some job's lattice has fourth-order slices
    bool mix_rb = false;       // some job's lattice has rectangular bends
    std::vector<const st_lattice*> lats;
    std::vector<int64_t> n, offset;
    std::vector<double> cost_per_particle;
    std::vector<uint8_t> uploaded;
    int64_t n_total = 0;
    double2 *xpx = nullptr, *ypy = nullptr, *tpt = nullptr, *sxy = nullptr;
    double* sz = nullptr;
    uint8_t* lost = nullptr;
    double* staging = nullptr;      // [9][max job n] for upload / download
    int64_t staging_n = 0;
    int32_t* status = nullptr;
    int32_t* queue = nullptr;       // device work-queue counter (scratch)
    JobDesc* d_jobs = nullptr;
    WorkItem* d_items = nullptr;
    int32_t n_items = 0;
    int32_t items_block = 0;
    size_t smem_bytes = 0;
    int32_t block_threads = 128;
    int32_t turns_per_launch = 5;
    int32_t use_graph = 1;
    int32_t variant = 0;   // the larger register budget: measured faster for both precisions
    cudaGraphExec_t graph = nullptr;
    int32_t g_turns = -1, g_K = -1, g_block = -1, g_tpl = -1, g_variant = -1;
};

static void batch_free(st_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->xpx);
    cudaFree(b->ypy);
    cudaFree(b->tpt);
    cudaFree(b->sxy);
    cudaFree(b->sz);
    cudaFree(b->lost);
    cudaFree(b->staging);
    cudaFree(b->status);
    cudaFree(b->queue);
    cudaFree(b->d_jobs);
    cudaFree(b->d_items);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Work items of `block` particles, largest estimated cost first.
static int build_items(st_batch* b, int block) {
    std::vector<WorkItem> items;
    std::vector<double> cost;
    for (int j = 0; j < b->n_jobs; ++j)
        for (int64_t f = 0; f < b->n[j]; f += block) {
            WorkItem w;
            w.job = j;
            w.first = (int32_t)(b->offset[j] + f);
            w.count = (int32_t)std::min<int64_t>(block, b->n[j] - f);
            w.pad_ = 0;
            items.push_back(w);
            cost.push_back(b->cost_per_particle[j] * w.count);
        }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return cost[a] > cost[c]; });
    std::vector<WorkItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    // items address particles by global index: make `first` relative to the job's arrays
    for (auto& w : sorted) w.first -= (int32_t)b->offset[w.job];
    cudaFree(b->d_items);
    b->d_items = nullptr;
    cudaError_t e = cudaMalloc(&b->d_items, sorted.size() * sizeof(WorkItem));
    if (e != cudaSuccess) return cuda_fail(e, "batch: work items");
    e = cudaMemcpy(b->d_items, sorted.data(), sorted.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch: work items copy");
    b->n_items = (int32_t)sorted.size();
    b->items_block = block;
    return ST_OK;
}

static int build_jobs(st_batch* b) {
    std::vector<JobDesc> jd(b->n_jobs);
    size_t smem = 0;
    for (int j = 0; j < b->n_jobs; ++j) {
        const LatticeImpl& L = b->lats[j]->impl;
        JobDesc d;
        memset(&d, 0, sizeof(d));
        if (b->precision == ST_FP64) {
            d.blob = L.d_blob;
            d.blob_bytes = (uint32_t)L.blob_bytes;
            d.seq_offset = (uint32_t)L.seq_offset;
            d.rho_offset = 0;
        } else {
            d.blob = L.d_mix;
            d.blob_bytes = (uint32_t)L.mix_bytes;
            d.seq_offset = (uint32_t)L.mix_seq_offset;
            d.rho_offset = (uint32_t)L.mix_rho_offset;
        }
        smem = std::max(smem, (size_t)d.blob_bytes);
        d.n_seq = L.n_elements;
        d.ref = L.ref;
        d.xpx = b->xpx + b->offset[j];
        d.ypy = b->ypy + b->offset[j];
        d.tpt = b->tpt + b->offset[j];
        d.sxy = b->sxy + b->offset[j];
        d.sz = b->sz + b->offset[j];
        d.lost = b->lost + b->offset[j];
        d.n = b->n[j];
        jd[j] = d;
    }
    if (smem > 200 * 1024) {
        set_error("batch: a lattice table of %zu bytes exceeds the 200 KiB shared-memory budget", smem);
        return ST_EINVAL;
    }
    b->smem_bytes = smem;
    cudaError_t e = cudaMalloc(&b->d_jobs, jd.size() * sizeof(JobDesc));
    if (e != cudaSuccess) return cuda_fail(e, "batch: job table");
    e = cudaMemcpy(b->d_jobs, jd.data(), jd.size() * sizeof(JobDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch: job table copy");
    return ST_OK;
}

// Kernel and grid for the current launch shape (no stream work; safe before a capture).
static int prepare_launch(st_batch* b, int K, BatchKernel* kern_out, int* grid_out) {
    BatchKernel kern =
        batch_kernel(b->precision, K, b->variant, b->has_ext, b->mix_fringe, b->mix_ext, b->mix_o4, b->mix_rb);
    cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "batch: cudaFuncSetAttribute");
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, b->block_threads, b->smem_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "batch: occupancy");
    if (per_sm < 1) {
        set_error("batch: block of %d threads does not fit on an SM", b->block_threads);
        return ST_EINVAL;
    }
    int grid = sms * per_sm;
    if (grid > b->n_items) grid = b->n_items;
    *kern_out = kern;
    *grid_out = grid;
    return ST_OK;
}

// Enqueue ceil(n_turns / tpl) x (queue reset, persistent kernel) on the stream.
static int enqueue_with(st_batch* b, BatchKernel kern, int grid, int n_turns) {
    for (int t = 0; t < n_turns; t += b->turns_per_launch) {
        const int nt = std::min(b->turns_per_launch, n_turns - t);
        cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(int32_t), b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch: queue reset");
        kern<<<grid, b->block_threads, b->smem_bytes, b->stream>>>(b->d_jobs, b->d_items, b->n_items, b->queue, nt,
                                                                   b->status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "batch: kernel launch");
    }
    return ST_OK;
}

static int enqueue_turns(st_batch* b, int n_turns, int K) {
    BatchKernel kern = nullptr;
    int grid = 0;
    int rc = prepare_launch(b, K, &kern, &grid);
    if (rc) return rc;
    return enqueue_with(b, kern, grid, n_turns);
}

extern "C" {

int st_batch_create(const st_lattice* const* lattices, const int64_t* n_particles, int32_t n_jobs, int32_t precision,
                    void* cuda_stream, st_batch** out) {
    if (!lattices || !n_particles || !out || n_jobs < 1) {
        set_error("st_batch_create: null pointer or n_jobs < 1");
        return ST_EINVAL;
    }
    if (precision != ST_FP64 && precision != ST_MIXED) {
        set_error("st_batch_create: precision must be ST_FP64 or ST_MIXED");
        return ST_EINVAL;
    }
    st_batch* b = new (std::nothrow) st_batch();
    if (!b) {
        set_error("st_batch_create: host allocation failed");
        return ST_ENOMEM;
    }
    b->n_jobs = n_jobs;
    b->precision = precision;
    int64_t total = 0, maxn = 0;
    for (int j = 0; j < n_jobs; ++j) {
        if (!lattices[j] || n_particles[j] < 1 || n_particles[j] > (1 << 30)) {
            delete b;
            set_error("st_batch_create: job %d needs a lattice and 1 <= n <= 2^30 particles", j);
            return ST_EINVAL;
        }
        b->lats.push_back(lattices[j]);
        if (lattices[j]->impl.has_ext) b->has_ext = true;
        if (lattices[j]->impl.mix_fringe) b->mix_fringe = true;
        if (lattices[j]->impl.mix_ext) b->mix_ext = true;
        if (lattices[j]->impl.mix_o4) b->mix_o4 = true;
        if (lattices[j]->impl.mix_rb) b->mix_rb = true;
        b->n.push_back(n_particles[j]);
        b->offset.push_back(total);
        total += n_particles[j];
        maxn = std::max(maxn, n_particles[j]);
        // cost per particle and turn: drifts 1, spin elements 6 per slice edge
        const LatticeImpl& L = lattices[j]->impl;
        double c = 0.0;
        for (int e = 0; e < L.n_elements; ++e) {
            const DevElem& d = L.h_table[L.h_seq[e]];
            c += is_spin_type(d.type) ? 6.0 * (d.n_slices + 1) : 1.0;
        }
        b->cost_per_particle.push_back(c);
    }
    if (total > ((int64_t)1 << 31) - 1) {   // the kernels index particles with int
        delete b;
        set_error("st_batch_create: at most 2^31 - 1 particles in total");
        return ST_EINVAL;
    }
    b->uploaded.assign(n_jobs, 0);
    b->n_total = total;
    b->staging_n = maxn;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "st_batch_create: stream");
        }
        b->own_stream = true;
    }
    const size_t N = (size_t)total;
#define ST_BALLOC(ptr, bytes)                                                                                     \
    e = cudaMalloc((void**)&(ptr), (bytes));                                                                      \
    if (e != cudaSuccess) {                                                                                       \
        batch_free(b);                                                                                            \
        set_error("st_batch_create: cudaMalloc of %zu bytes failed: %s", (size_t)(bytes), cudaGetErrorString(e)); \
        return ST_ENOMEM;                                                                                         \
    }
    ST_BALLOC(b->xpx, N * sizeof(double2));
    ST_BALLOC(b->ypy, N * sizeof(double2));
    ST_BALLOC(b->tpt, N * sizeof(double2));
    ST_BALLOC(b->sxy, N * sizeof(double2));
    ST_BALLOC(b->sz, N * sizeof(double));
    ST_BALLOC(b->lost, N);
    ST_BALLOC(b->staging, 9 * (size_t)maxn * sizeof(double));
    ST_BALLOC(b->status, sizeof(int32_t));
    ST_BALLOC(b->queue, sizeof(int32_t));
#undef ST_BALLOC
    e = cudaMemset(b->lost, 0, N);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "st_batch_create: init");
    }
    int rc = build_jobs(b);
    if (rc == ST_OK) rc = build_items(b, b->block_threads);
    if (rc != ST_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return ST_OK;
}

int st_batch_destroy(st_batch* b) {
    if (!b) return ST_OK;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    return ST_OK;
}

int st_batch_upload(st_batch* b, int32_t job, const double* z_soa, const double* spin_soa, int32_t src_is_device) {
    if (!b || !z_soa || !spin_soa || job < 0 || job >= b->n_jobs) {
        set_error("st_batch_upload: null pointer or job out of range");
        return ST_EINVAL;
    }
    const int64_t n = b->n[job], off = b->offset[job];
    cudaError_t e = cudaSuccess;
    const double *dz = z_soa, *ds = spin_soa;
    if (!src_is_device) {
        e = cudaMemcpyAsync(b->staging, z_soa, 6 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->staging + 6 * n, spin_soa, 3 * n * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "st_batch_upload: copy");
        dz = b->staging;
        ds = b->staging + 6 * n;
    }
    pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(dz, ds, b->xpx + off, b->ypy + off, b->tpt + off,
                                                                    b->sxy + off, b->sz + off, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(b->lost + off, 0, n, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_batch_upload");
    b->uploaded[job] = 1;
    return ST_OK;
}

int st_batch_set_launch(st_batch* b, int32_t block_threads, int32_t turns_per_launch, int32_t use_graph,
                        int32_t variant) {
    if (!b) {
        set_error("st_batch_set_launch: null batch");
        return ST_EINVAL;
    }
    if (block_threads != 0 && (block_threads < 32 || block_threads > 128 || block_threads % 32)) {
        set_error("st_batch_set_launch: block_threads must be a multiple of 32 in [32, 128]");
        return ST_EINVAL;
    }
    if (turns_per_launch < 0 || variant < -1 || variant > 1) {
        set_error("st_batch_set_launch: turns_per_launch >= 0, variant in {-1, 0, 1}");
        return ST_EINVAL;
    }
    if (block_threads && block_threads != b->items_block) {
        int rc = build_items(b, block_threads);
        if (rc) return rc;
    }
    if (block_threads) b->block_threads = block_threads;
    if (turns_per_launch) b->turns_per_launch = turns_per_launch;
    if (use_graph >= 0) b->use_graph = use_graph ? 1 : 0;
    if (variant >= 0) b->variant = variant;
    return ST_OK;
}

int st_batch_track(st_batch* b, int32_t n_turns, int32_t spin_order) {
    if (!b) {
        set_error("st_batch_track: null batch");
        return ST_EINVAL;
    }
    for (int j = 0; j < b->n_jobs; ++j)
        if (!b->uploaded[j]) {
            set_error("st_batch_track: job %d has no particles uploaded", j);
            return ST_ESTATE;
        }
    if (n_turns < 0 || spin_order < ST_SPIN_MID_KICK || spin_order > 4) {
        set_error("st_batch_track: need n_turns >= 0 and spin_order in -2..4");
        return ST_EINVAL;
    }
    if (spin_order < 0) {
        bool order4 = false;
        for (int j = 0; j < b->n_jobs; ++j) order4 = order4 || b->lats[j]->impl.has_order4;
        if (order4) {
            set_error("st_batch_track: the midpoint schemes need second-order slice maps");
            return ST_EINVAL;
        }
    }
    for (int j = 0; j < b->n_jobs; ++j)
        if (spin_order > b->lats[j]->impl.min_spin_slices_pow2) {
            set_error("st_batch_track: job %d: spin_order %d needs n_slices divisible by %d", j, spin_order,
                      1 << spin_order);
            return ST_EINVAL;
        }
    if (n_turns == 0) return ST_OK;
    if (!b->use_graph) return enqueue_turns(b, n_turns, spin_order);
    const bool hit = b->graph && b->g_turns == n_turns && b->g_K == spin_order && b->g_block == b->block_threads &&
                     b->g_tpl == b->turns_per_launch && b->g_variant == b->variant;
    cudaError_t e;
    if (!hit) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        // kernel attribute and grid are set up outside the capture
        BatchKernel kern = nullptr;
        int grid = 0;
        int rc = prepare_launch(b, spin_order, &kern, &grid);
        if (rc) return rc;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "st_batch_track: begin capture");
        rc = enqueue_with(b, kern, grid, n_turns);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "st_batch_track: end capture");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return cuda_fail(e, "st_batch_track: instantiate");
        }
        b->g_turns = n_turns;
        b->g_K = spin_order;
        b->g_block = b->block_threads;
        b->g_tpl = b->turns_per_launch;
        b->g_variant = b->variant;
    }
    e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_batch_track: graph launch");
    return ST_OK;
}

int st_batch_download(st_batch* b, int32_t job, double* spin_soa, double* z_soa, uint8_t* lost,
                      int32_t dst_is_device) {
    if (!b || !spin_soa || job < 0 || job >= b->n_jobs) {
        set_error("st_batch_download: null pointer or job out of range");
        return ST_EINVAL;
    }
    const int64_t n = b->n[job], off = b->offset[job];
    unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(
        b->staging, b->staging + 6 * n, b->xpx + off, b->ypy + off, b->tpt + off, b->sxy + off, b->sz + off, n);
    cudaError_t e = cudaGetLastError();
    cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(spin_soa, b->staging + 6 * n, 3 * n * sizeof(double), kind, b->stream);
    if (e == cudaSuccess && z_soa) e = cudaMemcpyAsync(z_soa, b->staging, 6 * n * sizeof(double), kind, b->stream);
    if (e == cudaSuccess && lost) e = cudaMemcpyAsync(lost, b->lost + off, n, kind, b->stream);
    int32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, b->status, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_batch_download");
    if (status == STATUS_BOUNDS) {
        set_error("st_batch_download: the checked build found an out-of-range table index or work item");
        return ST_EINVAL;
    }
    if (status != STATUS_OK) {
        set_error("st_batch_download: a batched kernel reported status %d (bounded wait expired)", status);
        return ST_ETIMEOUT;
    }
    return ST_OK;
}

int st_batch_autotune(st_batch* b, int32_t spin_order, int32_t trial_turns, int32_t* best_block, int32_t* best_tpl,
                      int32_t* best_variant, float* best_ms) {
    if (!b || trial_turns < 1) {
        set_error("st_batch_autotune: null batch or trial_turns < 1");
        return ST_EINVAL;
    }
    const size_t N = (size_t)b->n_total;
    const size_t bytes = N * (4 * sizeof(double2) + sizeof(double) + 1);
    unsigned char* backup = nullptr;
    cudaError_t e = cudaMalloc(&backup, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "st_batch_autotune: backup buffer");
    auto save = [&](bool restore) {
        unsigned char* p = backup;
        void* arr[6] = {b->xpx, b->ypy, b->tpt, b->sxy, b->sz, b->lost};
        size_t sz[6] = {N * sizeof(double2), N * sizeof(double2), N * sizeof(double2), N * sizeof(double2),
                        N * sizeof(double), N};
        cudaError_t ee = cudaSuccess;
        for (int k = 0; k < 6 && ee == cudaSuccess; ++k) {
            ee = restore ? cudaMemcpyAsync(arr[k], p, sz[k], cudaMemcpyDeviceToDevice, b->stream)
                         : cudaMemcpyAsync(p, arr[k], sz[k], cudaMemcpyDeviceToDevice, b->stream);
            p += sz[k];
        }
        return ee;
    };
    e = save(false);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks[3] = {64, 96, 128};
    const int tpls[2] = {1, trial_turns};
    float best = 1e30f;
    int bb = b->block_threads, bt = b->turns_per_launch, bv = b->variant;
    const int keep_graph = b->use_graph;
    b->use_graph = 0;
    int rc = (e == cudaSuccess) ? ST_OK : cuda_fail(e, "st_batch_autotune: setup");
    for (int ib = 0; ib < 3 && rc == ST_OK; ++ib)
        for (int it = 0; it < 2 && rc == ST_OK; ++it)
            for (int v = 0; v < 2 && rc == ST_OK; ++v) {
                rc = st_batch_set_launch(b, blocks[ib], tpls[it], -1, v);
                if (rc) break;
                rc = enqueue_turns(b, 1, spin_order);   // warm-up of this shape
                if (rc) break;
                cudaEventRecord(t0, b->stream);
                rc = enqueue_turns(b, trial_turns, spin_order);
                cudaEventRecord(t1, b->stream);
                if (rc) break;
                e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess) e = save(true);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "st_batch_autotune: trial");
                    break;
                }
                if (ms < best) {
                    best = ms;
                    bb = blocks[ib];
                    bt = tpls[it];
                    bv = v;
                }
            }
    b->use_graph = keep_graph;
    if (rc == ST_OK) rc = st_batch_set_launch(b, bb, bt, -1, bv);
    e = cudaStreamSynchronize(b->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(backup);
    if (rc == ST_OK && e != cudaSuccess) rc = cuda_fail(e, "st_batch_autotune");
    if (rc == ST_OK) {
        if (best_block) *best_block = bb;
        if (best_tpl) *best_tpl = bt;
        if (best_variant) *best_variant = bv;
        if (best_ms) *best_ms = best;
    }
    return rc;
}

}  // extern "C"
