// Slice-count tuner: the cheapest discretisation (base slice count n_b and
// spin scheme) of a lattice whose one-turn spin error stays within a bound.
//
// The paper chooses n_b and the number of Romberg iterations by comparing
// with a finely sliced reference (Sec. 5.2.1, 5.3: n_b = 128 or 256 with
// three iterations, error measure Delta S of Sec. 5.3).  This does the same
// on the GPU for a sample ensemble: every candidate (n_b, K) is tracked for
// one turn from the same state, its mean spin distance to the reference is
// measured, its turn is timed with CUDA events, and the fastest candidate
// within the bound is returned.  Host orchestration only: every turn runs in
// the FP64 tracker.
#include <cmath>
#include <cstring>
#include <vector>

#include "st_internal.cuh"

namespace st {

namespace {

struct TuneRun {
    std::vector<double> S;       // [3][n] spins after one turn
    std::vector<uint8_t> lost;   // [n]
    float ms = 0.0f;             // one timed turn
};

// One turn of the lattice with every spin-carrying element cut into nb
// slices, spin order K: state from the host arrays, one warm-up turn, one
// timed turn from the same state.
int tune_run(const std::vector<st_element>& base, const st_reference* ref, const double* z, const double* S,
             int64_t n, int nb, int K, TuneRun& out) {
    std::vector<st_element> els(base);
    for (auto& e : els)
        if (is_spin_type(e.type)) e.n_slices = nb;
    st_lattice* lat = nullptr;
    st_ctx* ctx = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int rc = st_lattice_create(els.data(), (int32_t)els.size(), ref, &lat);
    if (rc == ST_OK) rc = st_ctx_create(lat, n, ST_FP64, nullptr, &ctx);
    if (rc == ST_OK) rc = st_ctx_set_launch(ctx, 128, 1);
    if (rc == ST_OK) rc = st_particles_upload(ctx, z, S, 0);
    if (rc == ST_OK) rc = st_track(ctx, 1, K);
    if (rc == ST_OK) rc = st_particles_upload(ctx, z, S, 0);
    if (rc == ST_OK) {
        cudaError_t e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        if (e == cudaSuccess) e = cudaEventRecord(t0, ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_tune_slicing: events");
    }
    if (rc == ST_OK) rc = st_track(ctx, 1, K);
    if (rc == ST_OK) {
        cudaError_t e = cudaEventRecord(t1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&out.ms, t0, t1);
        if (e != cudaSuccess) rc = cuda_fail(e, "st_tune_slicing: timing");
    }
    if (rc == ST_OK) {
        out.S.assign(3 * (size_t)n, 0.0);
        out.lost.assign((size_t)n, 0);
        rc = st_spins_download(ctx, out.S.data(), nullptr, out.lost.data(), 0);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (ctx) st_ctx_destroy(ctx);
    if (lat) st_lattice_destroy(lat);
    return rc;
}

// Delta S (Sec. 5.3): mean |S_j - S_j(ref)| over the particles tracked in both.
double mean_spin_distance(const TuneRun& a, const TuneRun& r, int64_t n) {
    double sum = 0.0;
    int64_t m = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (a.lost[j] || r.lost[j]) continue;
        const double dx = a.S[j] - r.S[j], dy = a.S[n + j] - r.S[n + j], dz = a.S[2 * n + j] - r.S[2 * n + j];
        sum += std::sqrt(dx * dx + dy * dy + dz * dz);
        ++m;
    }
    return m ? sum / (double)m : 0.0;
}

}  // namespace

}  // namespace st

using namespace st;

extern "C" int st_tune_slicing(const st_element* elems, int32_t n_elems, const st_reference* ref, const double* z_soa,
                               const double* spin_soa, int64_t n_particles, double spin_error_bound,
                               int32_t* n_slices_out, int32_t* spin_order_out, double* dS_out, float* ms_out,
                               int32_t* n_candidates_out, double* table_out) {
    if (!elems || !ref || !z_soa || !spin_soa || !n_slices_out || !spin_order_out || n_elems < 1 ||
        n_particles < 1 || !(spin_error_bound > 0.0)) {
        set_error("st_tune_slicing: null pointer, empty input or non-positive bound");
        return ST_EINVAL;
    }
    for (int i = 0; i < n_elems; ++i) {
        if (const char* why = element_error(elems[i])) {
            set_error("st_tune_slicing: element %d: %s", i, why);
            return ST_EINVAL;
        }
    }
    const std::vector<st_element> base(elems, elems + n_elems);
    TuneRun ref_run;
    int rc = tune_run(base, ref, z_soa, spin_soa, n_particles, ST_TUNE_REF_SLICES, ST_TUNE_REF_ORDER, ref_run);
    if (rc != ST_OK) return rc;
    int best_nb = ST_TUNE_REF_SLICES, best_K = ST_TUNE_REF_ORDER, n_cand = 0;
    double best_dS = 0.0;
    float best_ms = ref_run.ms;
    for (int nb = 1; nb <= ST_TUNE_MAX_SLICES; nb *= 2) {
        for (int K = 0; K <= ST_TUNE_MAX_ORDER && (1 << K) <= nb; ++K) {
            TuneRun run;
            rc = tune_run(base, ref, z_soa, spin_soa, n_particles, nb, K, run);
            if (rc == ST_EINVAL) continue;   // a slicing the lattice does not admit (e.g. a TEAPOT
                                             // bend of 1 rad or more in one slice): not a candidate
            if (rc != ST_OK) return rc;
            const double dS = mean_spin_distance(run, ref_run, n_particles);
            if (table_out) {
                table_out[4 * n_cand + 0] = nb;
                table_out[4 * n_cand + 1] = K;
                table_out[4 * n_cand + 2] = dS;
                table_out[4 * n_cand + 3] = run.ms;
            }
            ++n_cand;
            if (dS <= spin_error_bound && run.ms < best_ms) {
                best_nb = nb;
                best_K = K;
                best_dS = dS;
                best_ms = run.ms;
            }
        }
    }
    *n_slices_out = best_nb;
    *spin_order_out = best_K;
    if (dS_out) *dS_out = best_dS;
    if (ms_out) *ms_out = best_ms;
    if (n_candidates_out) *n_candidates_out = n_cand;
    return ST_OK;
}
