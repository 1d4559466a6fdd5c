// C ABI of the spintrack library: lattice packing, contexts, state upload and
// download, and dispatch of the tracking kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "st_internal.cuh"

namespace st {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return ST_ECUDA;
}

bool is_spin_type(int t) {
    return t == ST_MULT || t == ST_QUAD_MK || t == ST_SBEND || t == ST_SOLENOID || t == ST_RBEND || t == ST_TEAPOT ||
           t == ST_THIN_MULT;
}

// Field checks of one element (every entry point that takes elements):
// nullptr if valid, else what is wrong.
const char* element_error(const st_element& e) {
    if (e.type < ST_DRIFT || e.type > ST_THIN_MULT) return "unknown type";
    if (e.type == ST_THIN_MULT) {
        if (e.L != 0.0 || e.n_slices < 1 || e.n_slices > 4096 || !std::isfinite(e.k1) || !std::isfinite(e.k2))
            return "thin lens needs L = 0, finite integrated strengths and 1 <= n_slices <= 4096";
        if (e.fringe || e.split_order == 4) return "thin lens has no fringe kicks and no fourth-order map";
    } else if (is_spin_type(e.type) && (!(e.L > 0.0) || e.n_slices < 1 || e.n_slices > 4096)) {
        return "spin-carrying element needs L > 0 and 1 <= n_slices <= 4096";
    }
    if (e.fringe != 0 && e.fringe != 1) return "fringe must be 0 or 1";
    if (e.fringe && (e.type == ST_DRIFT || e.type == ST_SNAKE))
        return "fringe kicks need a multipole, quadrupole, bend or solenoid";
    if ((e.split_order != 0 && e.split_order != 2 && e.split_order != 4) ||
        (e.split_order == 4 && e.type != ST_MULT && e.type != ST_QUAD_MK && e.type != ST_TEAPOT))
        return "split_order must be 0 or 2, or 4 for a multipole, matrix-kick quadrupole or TEAPOT bend";
    if (e.type == ST_DRIFT && !(e.L >= 0.0)) return "drift needs L >= 0";
    if (e.type == ST_RBEND &&
        (e.angle == 0.0 || e.eta == 0.0 || !std::isfinite(e.e1) || !(std::fabs(0.5 * e.angle + e.e1) < 1.5) ||
         !(std::fabs(-0.5 * e.angle + e.e1) < 1.5)))
        return "rectangular bend needs angle != 0, eta != 0 and face angles below 1.5 rad";
    if (e.type == ST_SBEND && (e.angle == 0.0 || e.eta == 0.0 || !std::isfinite(e.angle / e.L)))
        return "sector bend needs angle != 0 and eta != 0";
    if (e.type == ST_TEAPOT && (e.angle == 0.0 || !std::isfinite(e.eta) || !std::isfinite(e.angle / e.L) ||
                                !(std::fabs(e.angle / e.n_slices) < 1.0)))
        return "TEAPOT bend needs angle != 0 and less than 1 rad per slice";
    return nullptr;
}

// Precompute the per-element constants the kernels use (all in FP64).
DevElem pack_element(const st_element& e) {
    DevElem d;
    memset(&d, 0, sizeof(d));
    d.type = e.type;
    d.n_slices = (int16_t)(is_spin_type(e.type) ? e.n_slices : 1);
    d.flags = (e.fringe && e.type != ST_SOLENOID) ? ST_ELEM_FRINGE : 0;
    if (e.split_order == 4 && (e.type == ST_MULT || e.type == ST_QUAD_MK || e.type == ST_TEAPOT))
        d.flags |= ST_ELEM_ORDER4;
    switch (e.type) {
    case ST_DRIFT:
        d.ds = e.L;
        break;
    case ST_MULT:
        d.ds = e.L / e.n_slices;
        d.a[0] = e.k1;
        d.a[1] = e.k2;
        break;
    case ST_QUAD_MK:
        d.ds = e.L / e.n_slices;
        d.a[0] = e.k1;
        d.a[1] = std::fabs(e.k1);
        break;
    case ST_THIN_MULT:
        // integrated strengths; the slice is 1/N of the unit kick parameter
        d.ds = 1.0 / e.n_slices;
        d.a[0] = e.k1;
        d.a[1] = e.k2;
        break;
    case ST_TEAPOT:
        // curvature and field ratio; the second-order slice's curved drift
        // and kick lengths in the places of the fourth-order sub-steps
        d.ds = e.L / e.n_slices;
        d.a[0] = e.angle / e.L;
        d.a[1] = e.eta;
        d.a[2] = 0.5 * d.ds;
        d.a[4] = d.ds;
        break;
    default:
        break;
    }
    if (d.flags & ST_ELEM_ORDER4) {
        // Yoshida (1990): S2(x1 ds) S2(x0 ds) S2(x1 ds) is fourth order for a
        // symmetric second-order S2 when 2 x1 + x0 = 1 and 2 x1^3 + x0^3 = 0
        const double x1 = 1.0 / (2.0 - std::cbrt(2.0)), x0 = 1.0 - 2.0 * x1;
        d.a[2] = 0.5 * x1 * d.ds;
        d.a[3] = 0.5 * (x1 + x0) * d.ds;
        d.a[4] = x1 * d.ds;
        d.a[5] = x0 * d.ds;
    }
    switch (e.type) {
    case ST_SBEND: {
        d.ds = e.L / e.n_slices;
        double h = e.angle / e.L;
        d.a[0] = h;
        d.a[1] = e.eta;
        d.a[2] = std::cos(h * d.ds);
        d.a[3] = std::sin(h * d.ds);
        d.a[4] = 1.0 / (e.eta * h);
        d.a[5] = 1.0 / e.eta;
        break;
    }
    case ST_RBEND: {
        // Sec. 3.2: faces met at phi_in and phi_out, design field from
        // Px = sin(phi_in) -> sin(phi_out) over L (Eq. (rhob)), offsets of
        // Eqs. (Xoffset), (Toffset) (the latter as the arc length; the
        // kernel divides by beta0)
        d.ds = e.L / e.n_slices;
        const double phi_in = 0.5 * e.angle + e.e1, phi_out = -0.5 * e.angle + e.e1;
        const double sd = std::sin(phi_in) - std::sin(phi_out);
        d.a[0] = e.eta * sd / e.L;
        d.a[1] = phi_in;
        d.a[2] = -phi_out;
        d.a[3] = -e.L * (std::cos(phi_in) - std::cos(phi_out)) / sd;
        d.a[4] = e.L * (phi_in - phi_out) / sd;
        break;
    }
    case ST_SOLENOID:
        d.ds = e.L / e.n_slices;
        d.a[0] = e.k1;           // b0/(B rho)
        d.a[1] = 0.5 * e.k1;     // eta of Eq. (solenoid)
        d.a[2] = 0.25 * e.k1;    // half of eta: the vector potential in the middle of a fringe
        break;
    case ST_SNAKE: {
        double c = std::cos(0.5 * e.snake_mu), s = std::sin(0.5 * e.snake_mu);
        d.a[0] = c;
        d.a[1] = s * std::sin(e.snake_phi);
        d.a[2] = 0.0;
        d.a[3] = s * std::cos(e.snake_phi);
        break;
    }
    }
    return d;
}

static bool same_elem(const DevElem& a, const DevElem& b) { return memcmp(&a, &b, sizeof(DevElem)) == 0; }

}  // namespace st

using namespace st;

extern "C" {

const char* st_last_error(void) { return g_err; }

const char* st_version(void) { return "spintrack 0.1 (sm_103a)"; }

int st_lattice_create(const st_element* elems, int32_t n, const st_reference* ref, st_lattice** out) {
    if (!elems || !ref || !out || n < 1) {
        set_error("st_lattice_create: null pointer or n < 1");
        return ST_EINVAL;
    }
    if (n > 65535) {
        set_error("st_lattice_create: at most 65535 elements per turn (got %d)", n);
        return ST_EINVAL;
    }
    if (!(ref->G > 0.0) || !(ref->Ggamma0 > ref->G)) {
        set_error("st_lattice_create: need G > 0 and Ggamma0 > G (gamma0 > 1)");
        return ST_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        if (const char* why = element_error(elems[i])) {
            set_error("element %d: %s", i, why);
            return ST_EINVAL;
        }
    }
    st_lattice* lat = new (std::nothrow) st_lattice();
    if (!lat) {
        set_error("st_lattice_create: host allocation failed");
        return ST_ENOMEM;
    }
    LatticeImpl& L = lat->impl;
    L.ref.G = ref->G;
    L.ref.gamma0 = ref->Ggamma0 / ref->G;
    L.ref.beta0 = std::sqrt(1.0 - 1.0 / (L.ref.gamma0 * L.ref.gamma0));
    L.ref.inv_beta0 = 1.0 / L.ref.beta0;
    L.n_elements = n;

    std::vector<DevElem> uniq;
    std::vector<uint16_t> seq(n);
    int max_slices = 1;
    int min_pow2 = 30;
    for (int i = 0; i < n; ++i) {
        DevElem d = pack_element(elems[i]);
        int idx = -1;
        for (size_t u = 0; u < uniq.size(); ++u)
            if (same_elem(uniq[u], d)) { idx = (int)u; break; }
        if (idx < 0) {
            idx = (int)uniq.size();
            uniq.push_back(d);
        }
        seq[i] = (uint16_t)idx;
        if ((d.flags & ST_ELEM_ORDER4) || d.type == ST_RBEND || d.type == ST_TEAPOT || d.type == ST_THIN_MULT)
            L.has_ext = true;
        if (d.flags & ST_ELEM_ORDER4) L.has_order4 = true;
        if (is_spin_type(d.type)) {
            max_slices = std::max(max_slices, (int)d.n_slices);
            int p = 0;
            while (((d.n_slices >> p) & 1) == 0 && p < 30) ++p;
            min_pow2 = std::min(min_pow2, p);
        }
    }
    if (uniq.size() > 2048) {
        delete lat;
        set_error("st_lattice_create: more than 2048 distinct elements");
        return ST_EINVAL;
    }
    L.n_unique = (int)uniq.size();
    L.max_slices = max_slices;
    L.min_spin_slices_pow2 = min_pow2;
    L.table_bytes = uniq.size() * sizeof(DevElem);
    L.seq_offset = L.table_bytes;
    size_t seq_bytes = ((size_t)n * sizeof(uint16_t) + 15) & ~(size_t)15;
    L.blob_bytes = L.table_bytes + seq_bytes;
    std::vector<unsigned char> blob(L.blob_bytes, 0);
    memcpy(blob.data(), uniq.data(), L.table_bytes);
    memcpy(blob.data() + L.seq_offset, seq.data(), (size_t)n * sizeof(uint16_t));
    L.h_table = (DevElem*)malloc(L.table_bytes);
    L.h_seq = (uint16_t*)malloc((size_t)n * sizeof(uint16_t));
    if (!L.h_table || !L.h_seq) {
        free(L.h_table);
        free(L.h_seq);
        delete lat;
        set_error("st_lattice_create: host allocation failed");
        return ST_ENOMEM;
    }
    memcpy(L.h_table, uniq.data(), L.table_bytes);
    memcpy(L.h_seq, seq.data(), (size_t)n * sizeof(uint16_t));
    cudaError_t e = cudaMalloc(&L.d_blob, L.blob_bytes);
    if (e != cudaSuccess) {
        free(L.h_table);
        free(L.h_seq);
        delete lat;
        return cuda_fail(e, "st_lattice_create: cudaMalloc");
    }
    e = cudaMemcpy(L.d_blob, blob.data(), L.blob_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(L.d_blob);
        free(L.h_table);
        free(L.h_seq);
        delete lat;
        return cuda_fail(e, "st_lattice_create: cudaMemcpy");
    }
    int rc = build_mixed_tables(L);
    if (rc != ST_OK) {
        cudaFree(L.d_blob);
        free(L.h_table);
        free(L.h_seq);
        delete lat;
        return rc;
    }
    *out = lat;
    return ST_OK;
}

int st_lattice_destroy(st_lattice* lat) {
    if (!lat) return ST_OK;
    cudaFree(lat->impl.d_mix);
    cudaFree(lat->impl.d_blob);
    free(lat->impl.h_table);
    free(lat->impl.h_seq);
    delete lat;
    return ST_OK;
}

static void free_ctx(st_ctx* c) {
    cudaFree(c->xpx);
    cudaFree(c->ypy);
    cudaFree(c->tpt);
    cudaFree(c->sxy);
    cudaFree(c->sz);
    cudaFree(c->lost);
    cudaFree(c->staging);
    cudaFree(c->status);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int st_ctx_create(const st_lattice* lat, int64_t n_particles, int32_t precision, void* cuda_stream,
                  st_ctx** out) {
    if (!lat || !out || n_particles < 1) {
        set_error("st_ctx_create: null pointer or n_particles < 1");
        return ST_EINVAL;
    }
    if (precision != ST_FP64 && precision != ST_MIXED) {
        set_error("st_ctx_create: precision must be ST_FP64 or ST_MIXED");
        return ST_EINVAL;
    }
    if (n_particles > ((int64_t)1 << 31) - 1) {   // the kernels index particles with int
        set_error("st_ctx_create: at most 2^31 - 1 particles");
        return ST_EINVAL;
    }
    st_ctx* c = new (std::nothrow) st_ctx();
    if (!c) {
        set_error("st_ctx_create: host allocation failed");
        return ST_ENOMEM;
    }
    c->lat = lat;
    c->n = n_particles;
    c->precision = precision;
    size_t n = (size_t)n_particles;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "st_ctx_create: stream");
        }
        c->own_stream = true;
    }
#define ST_ALLOC(ptr, bytes)                                      \
    e = cudaMalloc((void**)&(ptr), (bytes));                      \
    if (e != cudaSuccess) {                                       \
        free_ctx(c);                                              \
        set_error("st_ctx_create: cudaMalloc of %zu bytes failed: %s", (size_t)(bytes), cudaGetErrorString(e)); \
        return ST_ENOMEM;                                         \
    }
    ST_ALLOC(c->xpx, n * sizeof(double2));
    ST_ALLOC(c->ypy, n * sizeof(double2));
    ST_ALLOC(c->tpt, n * sizeof(double2));
    ST_ALLOC(c->sxy, n * sizeof(double2));
    ST_ALLOC(c->sz, n * sizeof(double));
    ST_ALLOC(c->lost, n);
    ST_ALLOC(c->staging, 9 * n * sizeof(double));
    ST_ALLOC(c->status, sizeof(int32_t));
#undef ST_ALLOC
    e = cudaMemsetAsync(c->status, 0, sizeof(int32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->lost, 0, n, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "st_ctx_create: init");
    }
    *out = c;
    return ST_OK;
}

int st_ctx_destroy(st_ctx* ctx) {
    if (!ctx) return ST_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return ST_OK;
}

int st_ctx_set_launch(st_ctx* ctx, int32_t block_threads, int32_t turns_per_launch) {
    if (!ctx) {
        set_error("st_ctx_set_launch: null context");
        return ST_EINVAL;
    }
    if (block_threads != 0 && (block_threads < 32 || block_threads > 1024 || block_threads % 32)) {
        set_error("st_ctx_set_launch: block_threads must be a multiple of 32 in [32, 1024]");
        return ST_EINVAL;
    }
    if (turns_per_launch < 0) {
        set_error("st_ctx_set_launch: turns_per_launch must be >= 1 (0 keeps)");
        return ST_EINVAL;
    }
    if (block_threads) ctx->block_threads = block_threads;
    if (turns_per_launch) ctx->turns_per_launch = turns_per_launch;
    return ST_OK;
}

int st_particles_upload(st_ctx* ctx, const double* z_soa, const double* spin_soa, int32_t src_is_device) {
    if (!ctx || !z_soa || !spin_soa) {
        set_error("st_particles_upload: null pointer");
        return ST_EINVAL;
    }
    size_t n = (size_t)ctx->n;
    cudaError_t e;
    const double* dz = z_soa;
    const double* ds = spin_soa;
    if (!src_is_device) {
        e = cudaMemcpyAsync(ctx->staging, z_soa, 6 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->staging + 6 * n, spin_soa, 3 * n * sizeof(double), cudaMemcpyHostToDevice,
                                ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "st_particles_upload: copy");
        dz = ctx->staging;
        ds = ctx->staging + 6 * n;
    }
    int rc = launch_pack(ctx, dz, ds);
    if (rc) return rc;
    e = cudaMemsetAsync(ctx->lost, 0, n, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_particles_upload: lost flags");
    if (!src_is_device) {
        // host buffers are only guaranteed valid during the call
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "st_particles_upload: sync");
    }
    ctx->uploaded = true;
    return ST_OK;
}

int st_lost_upload(st_ctx* ctx, const uint8_t* lost, int32_t src_is_device) {
    if (!ctx || !lost) {
        set_error("st_lost_upload: null pointer");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_lost_upload: upload the particles first");
        return ST_ESTATE;
    }
    const size_t n = (size_t)ctx->n;
    cudaError_t e = cudaMemcpyAsync(ctx->lost, lost, n, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess && !src_is_device) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_lost_upload");
    return ST_OK;
}

// spin_order: a Romberg order 0..4 that every spin-carrying element's slice
// count admits, or a midpoint scheme on an FP64 context without fourth-order
// slice maps.
static bool spin_scheme_ok(const st_ctx* ctx, int spin_order, const char* who) {
    const LatticeImpl& L = ctx->lat->impl;
    if (spin_order < ST_SPIN_MID_KICK || spin_order > 4) {
        set_error("%s: spin_order must be a Romberg order 0..4 or a midpoint scheme (-1, -2)", who);
        return false;
    }
    if (spin_order < 0) {
        if (L.has_order4) {
            set_error("%s: the midpoint schemes need second-order slice maps", who);
            return false;
        }
        return true;
    }
    if (spin_order > L.min_spin_slices_pow2) {
        set_error("%s: spin_order %d needs every spin-carrying element's n_slices divisible by %d", who,
                  spin_order, 1 << spin_order);
        return false;
    }
    return true;
}

int st_track(st_ctx* ctx, int32_t n_turns, int32_t spin_order) {
    if (!ctx) {
        set_error("st_track: null context");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_track: no particles uploaded");
        return ST_ESTATE;
    }
    if (n_turns < 0) {
        set_error("st_track: need n_turns >= 0");
        return ST_EINVAL;
    }
    if (!spin_scheme_ok(ctx, spin_order, "st_track")) return ST_EINVAL;
    if (n_turns == 0) return ST_OK;
    if (ctx->precision == ST_FP64) return launch_track_fp64(ctx, n_turns, spin_order);
    return launch_track_mixed(ctx, n_turns, spin_order);
}

int st_track_orbit(st_ctx* ctx, int32_t n_turns) {
    if (!ctx) {
        set_error("st_track_orbit: null context");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_track_orbit: no particles uploaded");
        return ST_ESTATE;
    }
    if (n_turns < 0) {
        set_error("st_track_orbit: need n_turns >= 0");
        return ST_EINVAL;
    }
    if (n_turns == 0) return ST_OK;
    return ctx->precision == ST_MIXED ? launch_track_mixed_orbit(ctx, n_turns) : launch_track_orbit(ctx, n_turns);
}

int st_track_one_turn_map(st_ctx* ctx, int32_t spin_order, const double* q_ref, double* q_out) {
    if (!ctx || !q_ref || !q_out) {
        set_error("st_track_one_turn_map: null pointer");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_track_one_turn_map: no particles uploaded");
        return ST_ESTATE;
    }
    if (ctx->precision != ST_FP64) {
        set_error("st_track_one_turn_map: needs an FP64 context");
        return ST_EINVAL;
    }
    if (!spin_scheme_ok(ctx, spin_order, "st_track_one_turn_map")) return ST_EINVAL;
    return launch_track_turn_map(ctx, spin_order, q_out, q_ref);
}

int st_track_average(st_ctx* ctx, int32_t n_turns, int32_t spin_order, double* spin_sum) {
    if (!ctx || !spin_sum) {
        set_error("st_track_average: null pointer");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_track_average: no particles uploaded");
        return ST_ESTATE;
    }
    if (n_turns < 0) {
        set_error("st_track_average: needs n_turns >= 0");
        return ST_EINVAL;
    }
    if (!spin_scheme_ok(ctx, spin_order, "st_track_average")) return ST_EINVAL;
    if (n_turns == 0) return ST_OK;
    if (ctx->precision == ST_MIXED) return launch_track_mixed(ctx, n_turns, spin_order, spin_sum);
    return launch_track_average(ctx, n_turns, spin_order, spin_sum);
}

int st_spins_download(st_ctx* ctx, double* spin_soa, double* z_soa, uint8_t* lost, int32_t dst_is_device) {
    if (!ctx || !spin_soa) {
        set_error("st_spins_download: null pointer");
        return ST_EINVAL;
    }
    if (!ctx->uploaded) {
        set_error("st_spins_download: no particles uploaded");
        return ST_ESTATE;
    }
    size_t n = (size_t)ctx->n;
    int rc = launch_unpack(ctx, ctx->staging, ctx->staging + 6 * n);
    if (rc) return rc;
    cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(spin_soa, ctx->staging + 6 * n, 3 * n * sizeof(double), kind, ctx->stream);
    if (e == cudaSuccess && z_soa)
        e = cudaMemcpyAsync(z_soa, ctx->staging, 6 * n * sizeof(double), kind, ctx->stream);
    if (e == cudaSuccess && lost) e = cudaMemcpyAsync(lost, ctx->lost, n, kind, ctx->stream);
    int32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "st_spins_download");
    if (status == STATUS_BOUNDS) {
        set_error("st_spins_download: the checked build found an out-of-range element-table index");
        return ST_EINVAL;
    }
    if (status != STATUS_OK) {
        set_error("st_spins_download: a tracking kernel reported status %d (bounded wait expired)", status);
        return ST_ETIMEOUT;
    }
    return ST_OK;
}

}  // extern "C"
