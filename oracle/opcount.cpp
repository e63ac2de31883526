// Floating-point operation counts of the oracle's arithmetic (test infrastructure, like the
// rest of this directory: nothing on the product path uses it).
//
// The oracle's C source (hydro_oracle.c) is compiled a second time, as C++, with its `double`
// replaced by `counted`: a number type that performs every operation in IEEE double exactly
// as the plain build does and increments a counter for the operation's kind.  No arithmetic
// of the scheme is restated here, so the counts are those of the oracle's own evaluation order
// of section 4.1 (primitive recovery, MinBee interpolation, HLLC, AddFlux, the CFL signal),
// and the results equal the plain build's bit for bit.  Built single-threaded (the counters
// are plain globals).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

namespace {
enum { K_ADD, K_MUL, K_DIV, K_SQRT, K_CMP, K_MINMAX, K_ABS, K_NEG, K_KINDS };
unsigned long long g_ops[K_KINDS];
}  // namespace

struct counted {
    double v;
    counted() = default;
    constexpr counted(double x) : v(x) {}
    explicit operator double() const { return v; }
    counted &operator+=(counted b) { ++g_ops[K_ADD]; v += b.v; return *this; }
    counted &operator-=(counted b) { ++g_ops[K_ADD]; v -= b.v; return *this; }
    counted &operator*=(counted b) { ++g_ops[K_MUL]; v *= b.v; return *this; }
    counted &operator/=(counted b) { ++g_ops[K_DIV]; v /= b.v; return *this; }
};
static_assert(sizeof(counted) == sizeof(double), "counted must lay out as a double");

static inline counted operator+(counted a, counted b) { ++g_ops[K_ADD]; return a.v + b.v; }
static inline counted operator-(counted a, counted b) { ++g_ops[K_ADD]; return a.v - b.v; }
static inline counted operator*(counted a, counted b) { ++g_ops[K_MUL]; return a.v * b.v; }
static inline counted operator/(counted a, counted b) { ++g_ops[K_DIV]; return a.v / b.v; }
static inline counted operator-(counted a) { ++g_ops[K_NEG]; return -a.v; }
static inline bool operator<(counted a, counted b) { ++g_ops[K_CMP]; return a.v < b.v; }
static inline bool operator<=(counted a, counted b) { ++g_ops[K_CMP]; return a.v <= b.v; }
static inline bool operator>(counted a, counted b) { ++g_ops[K_CMP]; return a.v > b.v; }
static inline bool operator>=(counted a, counted b) { ++g_ops[K_CMP]; return a.v >= b.v; }
static inline bool operator==(counted a, counted b) { ++g_ops[K_CMP]; return a.v == b.v; }
static inline bool operator!=(counted a, counted b) { ++g_ops[K_CMP]; return a.v != b.v; }
static inline counted sqrt(counted a) { ++g_ops[K_SQRT]; return std::sqrt(a.v); }
static inline counted fabs(counted a) { ++g_ops[K_ABS]; return std::fabs(a.v); }
static inline counted fmin(counted a, counted b) { ++g_ops[K_MINMAX]; return std::fmin(a.v, b.v); }
static inline counted fmax(counted a, counted b) { ++g_ops[K_MINMAX]; return std::fmax(a.v, b.v); }
static inline bool isfinite(counted a) { return std::isfinite(a.v); }  // a check, not arithmetic
// boundary values of the analytic test solutions, not part of the per-cell method: not counted
static inline counted sin(counted a) { return std::sin(a.v); }
static inline counted cos(counted a) { return std::cos(a.v); }
static inline counted pow(counted a, counted b) { return std::pow(a.v, b.v); }

#define double counted
extern "C" {
#include "hydro_oracle.c"
}
#undef double

extern "C" {
// Counts since the last reset, by kind: add/sub, mul, div, sqrt, compare, min/max, abs, neg.
int oracle_opcount_kinds(void) { return K_KINDS; }
void oracle_opcount_reset(void) { memset(g_ops, 0, sizeof g_ops); }
void oracle_opcount_get(unsigned long long *out) {
    for (int k = 0; k < K_KINDS; ++k) out[k] = g_ops[k];
}
}
