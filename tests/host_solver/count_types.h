// count_types.h -- floating-point types that count their own arithmetic, for the host build of the
// solver headers (test and measurement infrastructure). CF wraps float and CD wraps double; every
// +, -, * and / and every square root, reciprocal square root and reciprocal adds one to the
// FP32 or FP64 tally (a product that the device fuses into an FMA is a multiply and an add here,
// so an FMA counts as 2); comparisons, negation, min, max and fabs count nothing; tenth_power
// counts 3 (a logarithm, a product, an exponential). Instantiating the solver's templates with
// these types gives the number of operations the algorithm performs as written, independent of
// how the compiler schedules them.
#pragma once

#include <cmath>
#include <type_traits>

namespace sblm {

struct FlopTally {
    unsigned long long f32 = 0, f64 = 0;
};
inline FlopTally g_tally;

#define SBLM_COUNTED_TYPE(NAME, REP, FIELD)                                                              \
    struct NAME {                                                                                        \
        REP v;                                                                                           \
        NAME() = default;                                                                                \
        template <typename S, typename = std::enable_if_t<std::is_arithmetic_v<S>>>                      \
        constexpr NAME(S x) : v((REP)x) {}                                                               \
    };                                                                                                   \
    inline NAME operator+(NAME a, NAME b) { ++g_tally.FIELD; return NAME(a.v + b.v); }                  \
    inline NAME operator-(NAME a, NAME b) { ++g_tally.FIELD; return NAME(a.v - b.v); }                  \
    inline NAME operator*(NAME a, NAME b) { ++g_tally.FIELD; return NAME(a.v * b.v); }                  \
    inline NAME operator/(NAME a, NAME b) { ++g_tally.FIELD; return NAME(a.v / b.v); }                  \
    inline NAME operator-(NAME a) { return NAME(-a.v); }                                                 \
    inline NAME& operator+=(NAME& a, NAME b) { a = a + b; return a; }                                    \
    inline NAME& operator-=(NAME& a, NAME b) { a = a - b; return a; }                                    \
    inline NAME& operator*=(NAME& a, NAME b) { a = a * b; return a; }                                    \
    inline bool operator<(NAME a, NAME b) { return a.v < b.v; }                                          \
    inline bool operator<=(NAME a, NAME b) { return a.v <= b.v; }                                        \
    inline bool operator>(NAME a, NAME b) { return a.v > b.v; }                                          \
    inline bool operator>=(NAME a, NAME b) { return a.v >= b.v; }                                        \
    inline bool operator==(NAME a, NAME b) { return a.v == b.v; }                                        \
    inline bool operator!=(NAME a, NAME b) { return a.v != b.v; }                                        \
    inline NAME sqrt_(NAME a) { ++g_tally.FIELD; return NAME(std::sqrt(a.v)); }                          \
    inline NAME rsqrt_(NAME a) { ++g_tally.FIELD; return NAME((REP)1 / std::sqrt(a.v)); }                \
    inline NAME rcp(NAME a) { ++g_tally.FIELD; return NAME((REP)1 / a.v); }                              \
    inline NAME fabs(NAME a) { return NAME(std::fabs(a.v)); }                                            \
    inline NAME fmin(NAME a, NAME b) { return NAME(std::fmin(a.v, b.v)); }                              \
    inline NAME fmax(NAME a, NAME b) { return NAME(std::fmax(a.v, b.v)); }                              \
    inline bool isfinite(NAME a) { return std::isfinite(a.v); }                                         \
    inline NAME tenth_power(NAME a) { g_tally.FIELD += 3; return NAME(std::exp((REP)0.1 * std::log(a.v))); }

SBLM_COUNTED_TYPE(CF, float, f32)
SBLM_COUNTED_TYPE(CD, double, f64)
#undef SBLM_COUNTED_TYPE

// the solver's tolerances of each counted type are those of the type it wraps (forward.cuh must be
// included before this header)
template <>
struct Tol<CF> : Tol<float> {};
template <>
struct Tol<CD> : Tol<double> {};
template <>
struct Eps<CF> : Eps<float> {};
template <>
struct Eps<CD> : Eps<double> {};

}  // namespace sblm
