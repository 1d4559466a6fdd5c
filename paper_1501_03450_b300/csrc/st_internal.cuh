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
    int16_t n_slices;
    int16_t flags;  // ST_ELEM_FRINGE: thin fringe spin kicks at both ends (mult, quad, sbend, teapot);
                    // ST_ELEM_ORDER4: fourth-order slice map (mult, quad, teapot; a[2..5] its sub-steps)
    double ds;      // slice length (drift: full length)
    double a[6];    // type-specific constants, see pack_element()
};
enum { ST_ELEM_FRINGE = 1, ST_ELEM_ORDER4 = 2 };
static_assert(sizeof(DevElem) == 64, "DevElem must be 64 bytes");

// a[] layout per type
//   ST_DRIFT   : (unused)
//   ST_MULT    : a0 = k1, a1 = k2
//   ST_QUAD_MK : a0 = k1, a1 = |k1|
//   (both, fourth-order map: a2 = x1 ds/2, a3 = (x1 + x0) ds/2, a4 = x1 ds,
//    a5 = x0 ds with Yoshida's x1 = 1/(2 - 2^(1/3)), x0 = 1 - 2 x1)
//   ST_SBEND   : a0 = h, a1 = eta, a2 = cos(h ds), a3 = sin(h ds),
//                a4 = 1/(eta h), a5 = 1/eta
//   ST_SNAKE   : a0..a3 = unit quaternion (scalar first)
//   ST_RBEND   : a0 = b1/(B rho), a1 = phi_entr, a2 = -phi_exit, a3 = X offset,
//                a4 = arc length of the reference orbit
//   ST_THIN_MULT: a0 = k1 L, a1 = k2 L (integrated), ds = 1/n_slices
//   ST_TEAPOT  : a0 = h, a1 = eta; second-order slice: a2 = ds/2 (curved
//                drifts), a4 = ds (kick); fourth-order: a2..a5 as ST_MULT's

// Reference-particle constants passed by value to the kernels.
struct RefConst {
    double G;
    double gamma0;
    double beta0;
    double inv_beta0;
};

// ---- mixed-precision tables ------------------------------------------------
// Spin reference constants of one edge weight w_j = 2^j ds / 2 (j = 0..5 covers
// the end and interior weights of every Romberg level for orders 0..4).
// alpha = w_j * Omega_ref_y, where Omega_ref is the precession vector of the
// on-axis, on-momentum particle (bends only; zero elsewhere).  C(u) =
// cos(sqrt(u)/2) and S(u) = sin(sqrt(u)/2)/sqrt(u); their Taylor coefficients
// about u0 = alpha^2 give the deviation of the edge rotation from the
// reference rotation without cancellation.
// Taylor terms of the edge-deviation functions: the n-th term is about
// (b_y/2)^n / n! for a deviation angle b_y, so 8 terms keep strong bends at
// high G gamma (b_y up to ~0.5 at the coarsest Romberg level) below 1e-12.
constexpr int MIX_TAYLOR = 8;

struct MixWeight {
    float alpha;
    float ch, sh;     // cos(alpha/2), sin(alpha/2)
    float cf, sf;     // cos(alpha), sin(alpha)
    float S0;         // S(alpha^2)
    float dC[MIX_TAYLOR];   // C(u0 + du) - C(u0) = sum_n dC[n] du^(n+1)
    float dS[MIX_TAYLOR];   // S(u0 + du) - S(u0) = sum_n dS[n] du^(n+1)
    float2 Ky;        // d e_y / d b_y at b = 0 (first-order coefficient), as (hi, lo)
    float Kq;         // coefficient of du in e_y beyond Ky: ch alpha dS[0] - sh dC[0]
    float du3;        // |du| below which the terms n >= 3 of dC, dS are below 2^-27 of the first
};

// Constants of a TEAPOT bend's curved drift over len (Sec. 3.6) for the
// mixed-precision kernel: sin(h len), (1 - cos(h len))/h, sin(h len)/h,
// 1 - cos(h len), (len - sin(h len)/h)/beta0 and sin(h len)/beta0, as (hi, lo).
struct MixCurvedDrift {
    float2 sn_ff, A1_ff, A2_ff, omc_ff, dT0_ff, snb0_ff;
};

// Per unique element, constants of the mixed-precision kernel.  First-order
// (linear) map coefficients are kept as compensated (hi, lo) float pairs so
// that no systematic FP32 rounding enters the linear optics; second-order
// terms use plain FP32.
struct __align__(16) MixElem {
    int32_t type;
    int32_t n_slices;
    float ds;                         // slice length (drift: full length)
    int32_t rho_off;                  // bends: offset (float2 units) of cos/sin(omr*i*ds), i = 0..N
    float2 ds_ff;                     // ds as (hi, lo); the drift length of a multipole's slice, 0 for a
                                      // thin lens (its kicks and edge weights use ds and the *ds fields)
    float2 k1ds_ff;                   // multipole: k1 ds; matrix-kick quadrupole: |k1| (as (hi, lo))
    float k1, k2;                     // multipole / quadrupole strengths (quadrupole: k2 = |k1|)
    float cbm1, sb;                   // bend: cos(h ds) - 1, sin(h ds)
    float h, eta, ieta, ieh;          // bend: h, eta, 1/eta, 1/(eta h)
    float dT_eta, omr;                // bend: (1 - 1/eta) ds / beta0; Omega_ref_y
    float2 sbieh_ff;                  // bend: sin(h ds)/(eta h) as (hi, lo)
    float2 ietads_ff;                 // bend: ds/eta as (hi, lo)
    float2 sb_ff;                     // bend: sin(h ds) as (hi, lo)
    float2 cbmieh_ff;                 // bend: (cos(h ds) - 1)/(eta h) as (hi, lo)
    float2 etah_ff;                   // bend: eta h as (hi, lo)
    float2 ome_ff;                    // bend: 1 - eta as (hi, lo)
    float2 k2h_ff;                    // multipole: k2 ds / 2 as (hi, lo)
    float2 k2ds_ff;                   // multipole: k2 ds as (hi, lo)
    float2 eh2_ff;                    // bend: eta h^2 as (hi, lo)
    float2 cbm1_ff;                   // bend: cos(h ds) - 1 as (hi, lo)
    float2 dTeta_ff;                  // bend: (1 - 1/eta) ds / beta0 as (hi, lo)
    float2 ieh_ff;                    // bend: 1/(eta h) as (hi, lo)
    float2 pad2_;
    // bend, half-slice constants of the midpoint spin schemes (as (hi, lo)):
    // sin(h ds/2), sin(h ds/2)/(eta h), cos(h ds/2) - 1, (cos(h ds/2) - 1)/(eta h),
    // ds/(2 eta), (1 - 1/eta) ds / (2 beta0)
    float2 sbh_ff, sbiehh_ff, cbm1h_ff, cbmiehh_ff, ietadsh_ff, dTetah_ff;
    // TEAPOT bend: curved drifts of ds/2 (the slice's) and ds/4 (half-slices of
    // the midpoint scheme), and the kick of the bend's field over ds:
    // eta h ds and eta h^2 ds, as (hi, lo)
    MixCurvedDrift td[2];
    float2 ehl_ff, ehlh_ff;
    // solenoid (Sec. 3.7, 4.4): ks = b0/(B rho), eta = ks/2 of the body map, ks/4
    // (the vector potential in the middle of a fringe), ks (1 + G), as (hi, lo)
    float2 ks_ff, seta_ff, setaf_ff, ks1G_ff;
    // fourth-order slice (Sec. 3.3, Yoshida's S2(x1 ds) S2(x0 ds) S2(x1 ds) with
    // adjacent half steps merged), as (hi, lo): the drift / linear-flow /
    // curved-drift lengths x1 ds/2 and (x1 + x0) ds/2, the kick / nonlinear-step
    // lengths x1 ds and x0 ds, and the multipole kicks over those lengths (k1 l,
    // k2 l/2, k2 l; a TEAPOT bend's eta h l and eta h^2 l in the first two)
    float2 o4_d_ff[2], o4_s_ff[2], o4_k1_ff[2], o4_k2h_ff[2], o4_k2_ff[2];
    float2 rq[4];                     // reference rotation over the element (bends, snakes), (hi, lo) per component
    MixWeight w[6];
    // rectangular bend (Sec. 3.2): the FP64 descriptor, tracked in FP64 inside the
    // mixed kernels
    DevElem d64;
};
static_assert(sizeof(MixElem) % 16 == 0, "MixElem must be a multiple of 16 bytes");
// MixElem::type bit of an element with thin fringe spin kicks at both ends
// (Sec. 4.5, Eq. (skfringe)); only the kernels instantiated for such lattices
// read it (the element kind is the low byte).
enum { ST_MIX_FRINGE = 0x100 };
// MixElem::type bit of an element with the fourth-order slice map (read by the
// extended instantiation only)
enum { ST_MIX_ORDER4 = 0x200 };

// Kernel status word values (written by bounded device waits).
enum : int32_t { STATUS_OK = 0, STATUS_TMA_TIMEOUT = 1, STATUS_BOUNDS = 3 };

// Checked build (compiled with -DST_CHECKED into a separate library): the
// trackers test every element-table index and the batch loop its work items
// before use; a violation writes STATUS_BOUNDS to the launch's status word and
// freezes the particle (no trap).  The release build compiles the tests out.
#ifdef ST_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

struct LatticeImpl {
    RefConst ref;
    int32_t n_elements;     // sequence length (elements per turn)
    int32_t n_unique;
    int32_t max_slices;
    int32_t min_spin_slices_pow2;  // largest k with every spin element divisible by 2^k
    bool mix_fringe = false;       // mixed table entries carry ST_MIX_FRINGE (thin fringe spin kicks)
    bool mix_ext = false;          // the lattice has TEAPOT bends, solenoids or fourth-order maps (the
                                   // mixed kernels' extended instantiation)
    bool mix_o4 = false;           // ... fourth-order maps (the extended instantiation with them)
    bool mix_rb = false;           // ... rectangular bends (the instantiation with their FP64 island)
    bool has_ext = false;          // fourth-order slice maps, rectangular or TEAPOT bends or thin lenses present
    bool has_order4 = false;       // fourth-order slice maps present
    // device copy: [DevElem table (n_unique)] [uint16 sequence (n_elements), padded]
    void* d_blob = nullptr;
    size_t blob_bytes = 0;
    size_t table_bytes = 0;
    size_t seq_offset = 0;
    // host copies for validation
    DevElem* h_table = nullptr;
    uint16_t* h_seq = nullptr;
    // mixed-precision blob: [MixElem (n_unique)] [uint16 sequence (n_elements), padded] [float2 rho table]
    void* d_mix = nullptr;
    size_t mix_bytes = 0;
    size_t mix_seq_offset = 0;
    size_t mix_rho_offset = 0;
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

// Function attributes (such as the dynamic shared-memory limit) apply per
// device, so launchers keep one "already set" flag per device ordinal.
constexpr int kMaxDeviceFlags = 64;
struct PerDeviceOnce {
    bool done[kMaxDeviceFlags] = {};
};
// Runs set() once per device for this flag set; returns ST_OK or an error
// code (the message is set).
template <class F>
inline int once_per_device(PerDeviceOnce& once, F&& set, const char* what) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (dev >= 0 && dev < kMaxDeviceFlags && once.done[dev]) return ST_OK;
    e = set();
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (dev >= 0 && dev < kMaxDeviceFlags) once.done[dev] = true;
    return ST_OK;
}
bool is_spin_type(int t);
DevElem pack_element(const st_element& e);
const char* element_error(const st_element& e);

// kernel launchers (track_fp64.cu, track_mixed.cu)
int launch_track_fp64(st_ctx* ctx, int n_turns, int spin_order);
int launch_track_orbit(st_ctx* ctx, int n_turns);
int launch_track_turn_map(st_ctx* ctx, int spin_order, double* q_out, const double* q_ref);
int launch_track_average(st_ctx* ctx, int n_turns, int spin_order, double* spin_sum);
int launch_track_mixed(st_ctx* ctx, int n_turns, int spin_order, double* spin_sum = nullptr);
int launch_track_mixed_orbit(st_ctx* ctx, int n_turns);
// mixed-precision table builder (mixed_tables.cu)
int build_mixed_tables(LatticeImpl& L);
int launch_pack(st_ctx* ctx, const double* z_soa, const double* spin_soa);
int launch_unpack(st_ctx* ctx, double* z_soa, double* spin_soa);
__global__ void pack_kernel(const double* __restrict__ z, const double* __restrict__ s, double2* xpx, double2* ypy,
                            double2* tpt, double2* sxy, double* sz, int64_t n);
__global__ void unpack_kernel(double* __restrict__ z, double* __restrict__ s, const double2* xpx, const double2* ypy,
                              const double2* tpt, const double2* sxy, const double* sz, int64_t n);

}  // namespace st
