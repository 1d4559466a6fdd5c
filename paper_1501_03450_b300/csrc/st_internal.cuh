// Internal definitions shared by the host runtime and the tracking kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "spintrack.h"

namespace st {

// Packed, deduplicated element descriptor as the kernels read it from shared
// memory (64 bytes, 16-byte aligned so the whole table moves with one bulk
// copy).  Per-type constants are precomputed on the host in FP64.
struct __align__(16) DevElem {
    int32_t type;
    int32_t n_slices;
    double ds;      // slice length (drift: full length)
    double a[6];    // type-specific constants, see pack_element()
};
static_assert(sizeof(DevElem) == 64, "DevElem must be 64 bytes");

// a[] layout per type
//   ST_DRIFT   : (unused)
//   ST_MULT    : a0 = k1, a1 = k2
//   ST_QUAD_MK : a0 = k1, a1 = |k1|
//   ST_SBEND   : a0 = h, a1 = eta, a2 = cos(h ds), a3 = sin(h ds),
//                a4 = 1/(eta h), a5 = 1/eta
//   ST_SNAKE   : a0..a3 = unit quaternion (scalar first)

// Reference-particle constants passed by value to the kernels.
struct RefConst {
    double G;
    double gamma0;
    double beta0;
    double inv_beta0;
};

// Per-element FP32 copy of the constants used by the mixed-precision kernel.
struct __align__(16) DevElemF {
    int32_t type;
    int32_t n_slices;
    float ds;
    float a[5];
};
static_assert(sizeof(DevElemF) == 32, "DevElemF must be 32 bytes");

// Kernel status word values (written by bounded device waits).
enum : int32_t { STATUS_OK = 0, STATUS_TMA_TIMEOUT = 1 };

struct LatticeImpl {
    RefConst ref;
    int32_t n_elements;     // sequence length (elements per turn)
    int32_t n_unique;
    int32_t max_slices;
    int32_t min_spin_slices_pow2;  // largest k with every spin element divisible by 2^k
    // device copy: [DevElem table (n_unique)] [uint16 sequence (n_elements), padded]
    void* d_blob = nullptr;
    size_t blob_bytes = 0;
    size_t table_bytes = 0;
    size_t seq_offset = 0;
    // host copies for validation and the mixed-precision table
    DevElem* h_table = nullptr;
    uint16_t* h_seq = nullptr;
    int32_t* h_slices = nullptr;   // per unique element
};

}  // namespace st

struct st_lattice {
    st::LatticeImpl impl;
};

struct st_ctx {
    const st_lattice* lat = nullptr;
    int64_t n = 0;
    int32_t precision = ST_FP64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool uploaded = false;
    int32_t block_threads = 128;
    int32_t turns_per_launch = 8;
    // FP64 state, pair-SoA
    double2* xpx = nullptr;
    double2* ypy = nullptr;
    double2* tpt = nullptr;
    double2* sxy = nullptr;
    double* sz = nullptr;
    uint8_t* lost = nullptr;
    double* staging = nullptr;   // [9][n] doubles for upload/download packing
    int32_t* status = nullptr;   // device status word
};

namespace st {

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// kernel launchers (track_fp64.cu)
int launch_track_fp64(st_ctx* ctx, int n_turns, int spin_order);
int launch_pack(st_ctx* ctx, const double* z_soa, const double* spin_soa);
int launch_unpack(st_ctx* ctx, double* z_soa, double* spin_soa);

}  // namespace st
