// Operation-counting build of the oracle -- TEST AND MEASUREMENT
// INFRASTRUCTURE ONLY (like oracle.c itself; the CUDA library never loads it).
//
// The oracle's source is compiled unchanged with its scalar `real` replaced
// by `counted`, a double that tallies every floating-point operation the
// oracle performs on particle data: additions and subtractions, multiplica-
// tions, divisions, and each special function (square root, sine/cosine,
// tangent, arcsine, hyperbolic sine/cosine).  Operations on plain doubles
// (per-element constants such as 0.5 * ds) are not counted.  Dividing the
// tallies of one tracking call by its particle-element passes gives the
// method's algorithmic work per pass as the paper's algorithm states it.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

namespace {
struct Tally {
    uint64_t add, mul, div, sqrt, sincos, tan, asin, hyp;
};
Tally g_tally;

struct counted {
    double v;
    counted() = default;
    counted(double x) : v(x) {}
};
static_assert(sizeof(counted) == sizeof(double), "counted must be layout-compatible with double");

inline counted operator+(counted a, counted b) { ++g_tally.add; return a.v + b.v; }
inline counted operator-(counted a, counted b) { ++g_tally.add; return a.v - b.v; }
inline counted operator*(counted a, counted b) { ++g_tally.mul; return a.v * b.v; }
inline counted operator/(counted a, counted b) { ++g_tally.div; return a.v / b.v; }
inline counted operator-(counted a) { return -a.v; }
inline counted& operator+=(counted& a, counted b) { a = a + b; return a; }
inline counted& operator-=(counted& a, counted b) { a = a - b; return a; }
inline counted& operator*=(counted& a, counted b) { a = a * b; return a; }
inline counted& operator/=(counted& a, counted b) { a = a / b; return a; }
inline double creal(counted a) { return a.v; }
inline double cimag(counted) { return 0.0; }
inline double creal(double a) { return a; }
inline double cimag(double) { return 0.0; }
inline counted sqrt(counted a) { ++g_tally.sqrt; return std::sqrt(a.v); }
inline counted sin(counted a) { ++g_tally.sincos; return std::sin(a.v); }
inline counted cos(counted a) { ++g_tally.sincos; return std::cos(a.v); }
inline counted tan(counted a) { ++g_tally.tan; return std::tan(a.v); }
inline counted asin(counted a) { ++g_tally.asin; return std::asin(a.v); }
inline counted sinh(counted a) { ++g_tally.hyp; return std::sinh(a.v); }
inline counted cosh(counted a) { ++g_tally.hyp; return std::cosh(a.v); }
using std::cbrt;
using std::cos;
using std::fabs;
using std::sin;
using std::sqrt;
using std::tan;
}  // namespace

#define ORACLE_OPCOUNT 1
#define ORACLE_REAL counted
#include "oracle.c"

extern "C" {
// Track as orc_track (z [6][n], S [3][n] as doubles; single thread) and return
// the tallies: out[0..7] = add, mul, div, sqrt, sin+cos, tan, asin, sinh+cosh.
int opc_track(const orc_element* els, int n_el, double G, double Ggamma0, long n, double* z, double* S,
              uint8_t* lost, int n_turns, int K, uint64_t* out) {
    g_tally = Tally{};
    int rc = orc_track(els, n_el, G, Ggamma0, n, reinterpret_cast<counted*>(z), reinterpret_cast<counted*>(S), lost,
                       n_turns, K, 1);
    const Tally t = g_tally;
    out[0] = t.add; out[1] = t.mul; out[2] = t.div; out[3] = t.sqrt;
    out[4] = t.sincos; out[5] = t.tan; out[6] = t.asin; out[7] = t.hyp;
    return rc;
}
}
