// overlap_class.cuh -- the overlap class floor(255 c / N) of a pixel count c
// in a composite of N members (the "overlap classes" of the Fig. 1 caption),
// computed without a hardware division.
//
// N is the same for every pixel of a render, so the division is by an
// invariant divisor and becomes a multiply-high and shifts, after Granlund
// and Montgomery, "Division by invariant integers using multiplication"
// (PLDI 1994), the unsigned case for 32-bit dividends: with l = ceil(log2 N),
// m = floor(2^32 (2^l - N) / N) + 1, s1 = min(l, 1), s2 = max(l - 1, 0) and
// t = umulhi(m, x), floor(x / N) = (t + ((x - t) >> s1)) >> s2 for every
// x < 2^32.  Here x = 255 c < 2^32 whenever N < 2^24 (c <= N); larger N take a
// 64-bit division.  A count above N (only possible in a composite that an
// underflow has already invalidated) is held at class 255, so the colour
// table is never indexed out of range.
//
// For N < 2^16 (every 16-bit plane) one multiply-high suffices: with
// M = ceil(255 2^k / N) = (255 2^k + r) / N, 0 <= r < N, and 255 c = q N + f,
// 0 <= f < N, floor(c M / 2^k) = q + floor((f + c r / 2^k) / N), which is q
// whenever c r < 2^k.  With c <= N that holds for k = 32 when N < 2^16, and
// M < 2^32 when N >= 256; for N < 256 take k = 16 (c r < 255^2 < 2^16).  So
// class = umulhi(min(c, N) << (32 - k), M), the count clamped to N first.
#pragma once

#include <stdint.h>

namespace cpt {

struct ClassDivisor {
    uint64_t n;      // members N
    uint32_t m;      // multiplier
    uint32_t s1;
    uint32_t s2;
    uint32_t wide;   // N >= 2^24: divide in 64 bits
    uint32_t narrow; // 1 <= N < 2^16: class = umulhi(min(c, N) << ns, nm)
    uint32_t nm;
    uint32_t ns;
};

__host__ __device__ inline ClassDivisor class_divisor(uint64_t n) {
    ClassDivisor d{n, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (n == 0) return d;
    if (n < (1u << 16)) {
        const uint32_t k = n >= 256 ? 32u : 16u;
        d.narrow = 1u;
        d.nm = (uint32_t)(((255ull << k) + n - 1) / n);   // ceil(255 2^k / N)
        d.ns = 32u - k;
    }
    if (n >= (1u << 24)) {
        d.wide = 1u;
        return d;
    }
    uint32_t l = 0;
    while ((uint64_t(1) << l) < n) ++l;                       // ceil(log2 n)
    d.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - n)) / n + 1);
    d.s1 = l < 1 ? l : 1;
    d.s2 = l > 1 ? l - 1 : 0;
    return d;
}

// The class when d.narrow is set (1 <= N < 2^16).
__device__ __forceinline__ uint32_t overlap_class_narrow(uint32_t c, const ClassDivisor &d) {
    return __umulhi(min(c, (uint32_t)d.n) << d.ns, d.nm);
}

__device__ __forceinline__ uint32_t overlap_class(uint32_t c, const ClassDivisor &d) {
    if (d.narrow) return overlap_class_narrow(c, d);
    if (d.n == 0) return 0;
    if (c >= d.n) return 255;
    if (d.wide) return (uint32_t)((255ull * c) / d.n);
    const uint32_t x = 255u * c;
    const uint32_t t = __umulhi(d.m, x);
    return (t + ((x - t) >> d.s1)) >> d.s2;
}

}  // namespace cpt
