// Allocation-free FP64 tracking entry point.
//
// For callers that cannot allocate device memory themselves or through this
// library: code that runs inside an allocator or memory pool that owns all of
// the device memory, plug-ins whose host process forbids extra allocations, or
// real-time loops where a cudaMalloc would stall or fragment the heap.  The
// caller passes the particle state in device buffers it already owns; the
// packed lattice table and the kernel status word live in one file-scope
// device array below, so the call allocates nothing.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; calls that overlap on the GPU (different streams, or
// different host threads) race on it.  It is held by every GPU that loads the
// library until the process exits.  On the host the lattice is packed into
// one static buffer (96 KiB, part of the library image, no heap) under a
// mutex, so concurrent host threads serialise their packing and copy.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "st_internal.cuh"

namespace st {

// lattice blob (table + sequence) followed by the 16-byte status slot
static constexpr size_t kNoAllocBlobMax = 64 * 1024;
static constexpr size_t kNoAllocBytes = kNoAllocBlobMax + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
static int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "st_track_fp64_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("st_track_fp64_noalloc: device ordinal %d out of range", dev);
        return ST_EINVAL;
    }
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "st_track_fp64_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ST_OK;
}

// True if p is memory the current device can address as device memory
// (device or managed allocations); host pointers, registered or not, are
// refused.  cudaPointerGetAttributes allocates nothing.
static bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // clear the non-sticky error of an unknown pointer
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host packing buffers: one per process, guarded by g_pack_mutex.
static unsigned char g_host_blob[kNoAllocBlobMax];
static uint16_t g_host_seq[16384];
static std::mutex g_pack_mutex;

}  // namespace st

using namespace st;

extern "C" int st_track_fp64_noalloc(const st_element* elems, int32_t n_elems, const st_reference* ref,
                                     double* state, uint8_t* lost, int64_t n_particles, int32_t n_turns,
                                     int32_t spin_order, void* cuda_stream) {
    if (!elems || !ref || !state || !lost || n_elems < 1 || n_particles < 1) {
        set_error("st_track_fp64_noalloc: null pointer, n_elems < 1 or n_particles < 1");
        return ST_EINVAL;
    }
    if (n_particles > ((int64_t)1 << 31) - 1 || n_elems > 16384) {
        set_error("st_track_fp64_noalloc: at most 2^31-1 particles and 16384 elements");
        return ST_EINVAL;
    }
    if (n_turns < 0 || spin_order < ST_SPIN_MID_KICK || spin_order > 4) {
        set_error("st_track_fp64_noalloc: need n_turns >= 0 and spin_order in -2..4");
        return ST_EINVAL;
    }
    if (!(ref->G > 0.0) || !(ref->Ggamma0 > ref->G)) {
        set_error("st_track_fp64_noalloc: need G > 0 and Ggamma0 > G");
        return ST_EINVAL;
    }
    // The state is read and written as pairs of doubles (16-byte accesses).
    if (((uintptr_t)state & 15) != 0) {
        set_error("st_track_fp64_noalloc: state must be 16-byte aligned");
        return ST_EINVAL;
    }
    if (!is_device_pointer(state) || !is_device_pointer(lost)) {
        set_error("st_track_fp64_noalloc: state and lost must be device (or managed) memory");
        return ST_EINVAL;
    }
    // Pack the lattice into the static host buffer (no heap allocation).
    std::lock_guard<std::mutex> pack_lock(g_pack_mutex);
    unsigned char* host_blob = g_host_blob;
    uint16_t* seq = g_host_seq;
    DevElem* table = (DevElem*)host_blob;
    const int max_unique = 512;
    int n_unique = 0;
    for (int i = 0; i < n_elems; ++i) {
        const st_element& e = elems[i];
        if (const char* why = element_error(e)) {
            set_error("st_track_fp64_noalloc: element %d: %s", i, why);
            return ST_EINVAL;
        }
        if (is_spin_type(e.type) && spin_order > 0 && e.n_slices % (1 << spin_order) != 0) {
            set_error("st_track_fp64_noalloc: element %d: n_slices not a multiple of 2^spin_order", i);
            return ST_EINVAL;
        }
        if (spin_order < 0 && e.split_order == 4) {
            set_error("st_track_fp64_noalloc: element %d: the midpoint schemes need second-order slice maps", i);
            return ST_EINVAL;
        }
        DevElem d = pack_element(e);
        int idx = -1;
        for (int u = 0; u < n_unique; ++u)
            if (memcmp(&table[u], &d, sizeof(DevElem)) == 0) {
                idx = u;
                break;
            }
        if (idx < 0) {
            if (n_unique == max_unique) {
                set_error("st_track_fp64_noalloc: more than %d distinct elements", max_unique);
                return ST_EINVAL;
            }
            idx = n_unique++;
            table[idx] = d;
        }
        seq[i] = (uint16_t)idx;
    }
    const size_t table_bytes = (size_t)n_unique * sizeof(DevElem);
    const size_t seq_bytes = (((size_t)n_elems * sizeof(uint16_t)) + 15) & ~(size_t)15;
    if (table_bytes + seq_bytes > kNoAllocBlobMax) {
        set_error("st_track_fp64_noalloc: lattice needs %zu bytes, the scratch holds %zu",
                  table_bytes + seq_bytes, kNoAllocBlobMax);
        return ST_EINVAL;
    }
    memcpy(host_blob + table_bytes, seq, (size_t)n_elems * sizeof(uint16_t));
    memset(host_blob + table_bytes + (size_t)n_elems * sizeof(uint16_t), 0,
           seq_bytes - (size_t)n_elems * sizeof(uint16_t));

    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int32_t* status = (int32_t*)((unsigned char*)scratch + kNoAllocBlobMax);
    cudaError_t e = cudaMemcpyAsync(scratch, host_blob, table_bytes + seq_bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_track_fp64_noalloc: staging the lattice");

    if (n_turns > 0) {
        // Lattice and context views on the stack over the scratch and the
        // caller's buffers; the regular FP64 launcher does the rest.
        st_lattice lat;
        LatticeImpl& L = lat.impl;
        L.ref.G = ref->G;
        L.ref.gamma0 = ref->Ggamma0 / ref->G;
        L.ref.beta0 = sqrt(1.0 - 1.0 / (L.ref.gamma0 * L.ref.gamma0));
        L.ref.inv_beta0 = 1.0 / L.ref.beta0;
        L.n_elements = n_elems;
        L.n_unique = n_unique;
        L.d_blob = scratch;
        L.blob_bytes = table_bytes + seq_bytes;
        L.table_bytes = table_bytes;
        L.seq_offset = table_bytes;
        for (int u = 0; u < n_unique; ++u)
            if ((table[u].flags & ST_ELEM_ORDER4) || table[u].type == ST_RBEND || table[u].type == ST_TEAPOT ||
                table[u].type == ST_THIN_MULT)
                L.has_ext = true;
        st_ctx ctx;
        ctx.lat = &lat;
        ctx.n = n_particles;
        ctx.precision = ST_FP64;
        ctx.stream = stream;
        ctx.uploaded = true;
        ctx.block_threads = 128;
        ctx.turns_per_launch = 8;
        const size_t n = (size_t)n_particles;
        double2* pairs = (double2*)state;
        ctx.xpx = pairs;
        ctx.ypy = pairs + n;
        ctx.tpt = pairs + 2 * n;
        ctx.sxy = pairs + 3 * n;
        ctx.sz = state + 8 * n;
        ctx.lost = lost;
        ctx.status = status;
        rc = launch_track_fp64(&ctx, n_turns, spin_order);
        L.d_blob = nullptr;      // the views own nothing
        ctx.xpx = ctx.ypy = ctx.tpt = ctx.sxy = nullptr;
        ctx.sz = nullptr;
        ctx.lost = nullptr;
        ctx.status = nullptr;
        if (rc) return rc;
    }
    int32_t host_status = 0;
    e = cudaMemcpyAsync(&host_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_track_fp64_noalloc");
    if (host_status == STATUS_BOUNDS) {
        set_error("st_track_fp64_noalloc: the checked build found an out-of-range element-table index");
        return ST_EINVAL;
    }
    if (host_status != STATUS_OK) {
        set_error("st_track_fp64_noalloc: the tracking kernel reported status %d (bounded wait expired)",
                  host_status);
        return ST_ETIMEOUT;
    }
    return ST_OK;
}
