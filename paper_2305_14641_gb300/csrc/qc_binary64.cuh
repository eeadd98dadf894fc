// Binary64 addition of non-negative operands on the integer pipe.  GB300
// issues binary64 operations at a small fraction of its integer rate, so a hot
// loop that must round exactly like IEEE binary64 (round to nearest, ties to
// even) adds here.  Operands and results are bit patterns; non-negative
// binary64 values order like those integers.  Subnormal and infinite operands
// go to the hardware instruction, so every result equals the IEEE one.
// (A multiplier built the same way for the hop-distance potential was bit-exact
// but gained nothing measurable there: that kernel is not bound by binary64
// issue.)
#pragma once

#include <cstdint>

namespace qcfp {

constexpr unsigned long long MANT = (1ull << 52) - 1, IMPL = 1ull << 52;
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ull;

__device__ __forceinline__ double as_double(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ unsigned long long bits_of(double x) { return (unsigned long long)__double_as_longlong(x); }

// a + b.  Mantissas carry three extra bits (guard, round and a sticky bit that
// collects everything shifted out), the standard construction for a correctly
// rounded sum.
__device__ __forceinline__ unsigned long long add_pos(unsigned long long a, unsigned long long b) {
    if (a < b) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
    if (b == 0) return a;
    const int ea = (int)(a >> 52), eb = (int)(b >> 52);
    if (ea == 2047 || eb == 0) return bits_of(__dadd_rn(as_double(a), as_double(b)));
    const int d = ea - eb;
    if (d >= 54) return a;                      // b is below half an ulp of a
    const unsigned long long ma = ((a & MANT) | IMPL) << 3;
    const unsigned long long mb0 = ((b & MANT) | IMPL) << 3;
    const unsigned long long mb = (mb0 >> d) | (unsigned long long)((mb0 & ((1ull << d) - 1)) != 0);
    unsigned long long s = ma + mb;             // below 2^57
    int e = ea;
    if (s >> 56) {
        s = (s >> 1) | (s & 1ull);
        ++e;
    }
    const unsigned low = (unsigned)(s & 7ull);
    s >>= 3;
    if (low > 4u || (low == 4u && (s & 1ull))) ++s;
    if (s >> 53) {
        s >>= 1;
        ++e;
    }
    if (e >= 2047) return INF_BITS;
    return ((unsigned long long)e << 52) | (s & MANT);
}

}  // namespace qcfp
