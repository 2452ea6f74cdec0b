// Hermitian half layout (M = 2 and M = 3): index decoding and conjugation helpers shared by the
// single-instance kernels and the batched kernel.
//
// Swapping the forward and backward path of every point (x = (s+, s-) -> (s-, s+), digit
// values 1 <-> 2) conjugates K and every influence factor (Sec. II, Eqs. for K and I), so a
// Hermitian rho(0) gives A(conj x) = conj(A(x)) at every step.  A prefix is canonical when
// its most significant digit outside {0, 3} is a 1; canonical n-digit prefixes are ordered
// [top 1: 4^(n-1) plain][top 0: canonical n-1][top 3: canonical n-1], C(n) = (4^n + 2^n)/2
// of them.  An n-digit tensor stores the 4-entry last-digit fiber of every canonical
// (n-1)-digit prefix, prefix c at entry 4c.
#pragma once

#include "quapi_internal.h"

namespace quapi {

__host__ __device__ __forceinline__ int64_t half_count(int n) {  // C(n)
    return ((int64_t(1) << (2 * n)) + (int64_t(1) << n)) >> 1;
}
__host__ __device__ __forceinline__ int64_t half_entries(int n) {  // stored entries of n digits
    return n == 0 ? 1 : 4 * half_count(n - 1);
}

// canonical position c among n-digit prefixes -> plain digits and whether the
// prefix is its own conjugate (all digits 0 or 3).  32-bit: n <= 15.
__device__ __forceinline__ uint32_t half_count32(int n) { return ((1u << (2 * n)) + (1u << n)) >> 1; }

__device__ __forceinline__ void half_decode(uint32_t c, int n, uint32_t& plain, bool& sc) {
    uint32_t p = 0;
    for (int level = n; level >= 1; --level) {
        const uint32_t r1 = 1u << (2 * (level - 1));
        if (c < r1) {  // digit 1, the rest is plain
            plain = (p << (2 * level)) | r1 | c;
            sc = false;
            return;
        }
        c -= r1;
        const uint32_t cn1 = half_count32(level - 1);
        if (c < cn1) {
            p = p << 2;
        } else {
            c -= cn1;
            p = (p << 2) | 3u;
        }
    }
    plain = p;
    sc = true;
}

// half_decode together with the prefix fh = f >> 2 (f without its last digit,
// n - 1 digits): its canonical position h and whether it is its own conjugate.
// The digits above f's first digit 1 are shared with fh, so one walk down the
// levels gives both positions (fh of a canonical f is canonical).
__device__ __forceinline__ void half_decode_pair(uint32_t c, int n, uint32_t& plain, bool& sc, uint32_t& h,
                                                 bool& shc) {
    uint32_t p = 0, hoff = 0;
    for (int level = n; level >= 1; --level) {
        const uint32_t r1 = 1u << (2 * (level - 1));
        if (c < r1) {  // digit 1 at this level, the rest is plain
            plain = (p << (2 * level)) | r1 | c;
            sc = false;
            h = hoff + (c >> 2);      // level >= 2: fh keeps the digit 1 and the plain rest c >> 2
            shc = (level == 1);       // level 1: the digit 1 was f's last digit, fh is all 0s and 3s
            return;
        }
        c -= r1;
        const uint32_t cn1 = half_count32(level - 1);
        // fh's layout at level - 1: [digit 1: r1 / 4][digit 0: C(level - 2)][digit 3: C(level - 2)]
        const uint32_t skip = (level >= 2) ? (r1 >> 2) : 0u;
        if (c < cn1) {
            p = p << 2;
            hoff += skip;
        } else {
            c -= cn1;
            p = (p << 2) | 3u;
            hoff += (level >= 2) ? skip + half_count32(level - 2) : 0u;
        }
    }
    plain = p;
    sc = true;
    h = hoff;
    shc = true;
}

// canonical position of a canonical n-digit prefix given by its plain digits
__device__ __forceinline__ uint32_t half_position(uint32_t h, int n) {
    uint32_t idx = 0;
    for (int level = n; level >= 1; --level) {
        const uint32_t d = (h >> (2 * (level - 1))) & 3u;
        const uint32_t r1 = 1u << (2 * (level - 1));
        if (d == 1u) return idx + (h & (r1 - 1u));
        idx += r1;
        if (d == 3u) idx += half_count32(level - 1);
    }
    return idx;
}

__device__ __forceinline__ bool self_conjugate(uint32_t h, int n) {  // every digit 0 or 3
    const uint32_t mask = (n >= 16) ? 0x55555555u : ((1u << (2 * n)) - 1u) & 0x55555555u;
    return ((h ^ (h >> 1)) & mask) == 0u;
}

__device__ __forceinline__ uint32_t conj_digits(uint32_t f) {
    return ((f & 0x55555555u) << 1) | ((f & 0xAAAAAAAAu) >> 1);
}

// ---- M = 3 ---------------------------------------------------------------------------------
// Points x = 3a + b (a, b = 0..2); conjugation (a, b) -> (b, a) swaps 1 <-> 3, 2 <-> 6, 5 <-> 7 and
// keeps the self-conjugate 0, 4, 8.  A prefix is canonical when its most significant digit that is
// not 0, 4 or 8 is 1, 2 or 5; canonical n-digit prefixes are ordered [top 1: 9^(n-1) plain][top 2:
// 9^(n-1) plain][top 5: 9^(n-1) plain][top 0: canonical n-1][top 4: canonical n-1][top 8: canonical
// n-1], C3(n) = (9^n + 3^n) / 2 of them; an n-digit tensor stores the 9-entry last-digit fiber of
// every canonical (n-1)-digit prefix, prefix c at entry 9c.  Indices are base-9 numbers in 32 bits
// (n <= 10 digits).
__host__ __device__ __forceinline__ uint32_t pow9(int k) {
    uint32_t r = 1;
    for (int i = 0; i < k; ++i) r *= 9u;
    return r;
}
__host__ __device__ __forceinline__ uint32_t half3_count(int n) {  // C3(n)
    uint32_t a = 1, b = 1;
    for (int i = 0; i < n; ++i) {
        a *= 9u;
        b *= 3u;
    }
    return (a + b) >> 1;
}
__host__ __device__ __forceinline__ int64_t half3_entries(int n) { return n == 0 ? 1 : 9 * (int64_t)half3_count(n - 1); }
__host__ __device__ __forceinline__ uint32_t top3_digit(uint32_t t) { return t == 0 ? 1u : (t == 1 ? 2u : 5u); }
__host__ __device__ __forceinline__ uint32_t conj3(uint32_t d) { return (d % 3u) * 3u + d / 3u; }
__host__ __device__ __forceinline__ bool self3(uint32_t d) { return d == 0u || d == 4u || d == 8u; }
// index of a canonical point among (1, 2, 5)
__host__ __device__ __forceinline__ uint32_t top3_index(uint32_t d) { return d == 1u ? 0u : (d == 2u ? 1u : 2u); }

// canonical position c among n-digit prefixes -> plain digits and whether the prefix is its own conjugate
__host__ __device__ __forceinline__ void half3_decode(uint32_t c, int n, uint32_t& plain, bool& sc) {
    uint32_t p = 0, P = pow9(n > 0 ? n - 1 : 0);
    for (int level = n; level >= 1; --level) {
        if (c < 3u * P) {
            const uint32_t t = c / P, rest = c - t * P;
            plain = (p * 9u + top3_digit(t)) * P + rest;
            sc = false;
            return;
        }
        c -= 3u * P;
        const uint32_t cn1 = half3_count(level - 1);
        const uint32_t t = c / cn1;
        c -= t * cn1;
        p = p * 9u + 4u * t;  // self-conjugate digits 0, 4, 8
        P /= 9u;
    }
    plain = p;
    sc = true;
}

// half3_decode together with the canonical position h of fh = f / 9 (the prefix without its last digit,
// n - 1 digits) and whether fh is its own conjugate (shc)
__host__ __device__ __forceinline__ void half3_decode_pair(uint32_t c, int n, uint32_t& plain, bool& sc, uint32_t& h,
                                                           bool& shc) {
    uint32_t p = 0, hoff = 0, P = pow9(n > 0 ? n - 1 : 0);
    for (int level = n; level >= 1; --level) {
        if (c < 3u * P) {
            const uint32_t t = c / P, rest = c - t * P;
            plain = (p * 9u + top3_digit(t)) * P + rest;
            sc = false;
            if (level >= 2) {  // fh keeps this digit: its block at fh's level has 9^(level-2) entries
                h = hoff + t * (P / 9u) + rest / 9u;
                shc = false;
            } else {  // the canonical digit was f's last one: fh is made of self-conjugate digits
                h = hoff;
                shc = true;
            }
            return;
        }
        c -= 3u * P;
        const uint32_t cn1 = half3_count(level - 1);
        const uint32_t t = c / cn1;
        c -= t * cn1;
        p = p * 9u + 4u * t;
        // fh's layout at level - 1: [3 top blocks of 9^(level-2)][self-conjugate blocks of C3(level-2)]
        if (level >= 2) hoff += 3u * (P / 9u) + t * half3_count(level - 2);
        P /= 9u;
    }
    plain = p;
    sc = true;
    h = hoff;
    shc = true;
}

// half3_decode_pair, and run = how many consecutive positions from c stay in the same plain block of a
// canonical top digit at level >= 2 (0 otherwise).  Position c + i (i < run) then has the prefix
// plain + i and its fh = (plain + i) / 9 the canonical position h + (plain % 9 + i) / 9.
__host__ __device__ __forceinline__ void half3_decode_run(uint32_t c, int n, uint32_t& plain, bool& sc, uint32_t& h,
                                                          bool& shc, uint32_t& run) {
    uint32_t p = 0, hoff = 0, P = pow9(n > 0 ? n - 1 : 0);
    run = 0;
    for (int level = n; level >= 1; --level) {
        if (c < 3u * P) {
            const uint32_t t = c / P, rest = c - t * P;
            plain = (p * 9u + top3_digit(t)) * P + rest;
            sc = false;
            if (level >= 2) {
                h = hoff + t * (P / 9u) + rest / 9u;
                shc = false;
                run = P - rest;
            } else {
                h = hoff;
                shc = true;
            }
            return;
        }
        c -= 3u * P;
        const uint32_t cn1 = half3_count(level - 1);
        const uint32_t t = c / cn1;
        c -= t * cn1;
        p = p * 9u + 4u * t;
        if (level >= 2) hoff += 3u * (P / 9u) + t * half3_count(level - 2);
        P /= 9u;
    }
    plain = p;
    sc = true;
    h = hoff;
    shc = true;
}

// canonical position of a canonical n-digit prefix given by its plain digits
__host__ __device__ __forceinline__ uint32_t half3_position(uint32_t hp, int n) {
    uint32_t idx = 0, P = pow9(n > 0 ? n - 1 : 0);
    for (int level = n; level >= 1; --level) {
        const uint32_t d = (hp / P) % 9u;
        if (!self3(d)) return idx + top3_index(d) * P + hp % P;
        idx += 3u * P + (d / 4u) * half3_count(level - 1);
        P /= 9u;
    }
    return idx;
}

__host__ __device__ __forceinline__ bool self_conjugate3(uint32_t hp, int n) {
    for (int i = 0; i < n; ++i, hp /= 9u)
        if (!self3(hp % 9u)) return false;
    return true;
}

__host__ __device__ __forceinline__ uint32_t conj_digits3(uint32_t f, int n) {
    uint32_t r = 0, scale = 1;
    for (int i = 0; i < n; ++i, f /= 9u, scale *= 9u) r += conj3(f % 9u) * scale;
    return r;
}

__device__ __forceinline__ double2 conjv(double2 v) { return make_double2(v.x, -v.y); }
__device__ __forceinline__ float2 conjv(float2 v) { return make_float2(v.x, -v.y); }
__device__ __forceinline__ df2 conjv(df2 v) {
    v.h.y = -v.h.y;
    v.l.y = -v.l.y;
    return v;
}
__device__ __forceinline__ double2 twice_real(double2 v) { return make_double2(2.0 * v.x, 0.0); }
__device__ __forceinline__ float2 twice_real(float2 v) { return make_float2(2.f * v.x, 0.f); }
__device__ __forceinline__ df2 twice_real(df2 v) {
    v.h = make_float2(2.f * v.h.x, 0.f);
    v.l = make_float2(2.f * v.l.x, 0.f);
    return v;
}
__device__ __forceinline__ double2 real_part(double2 v) { return make_double2(v.x, 0.0); }
__device__ __forceinline__ float2 real_part(float2 v) { return make_float2(v.x, 0.f); }
__device__ __forceinline__ df2 real_part(df2 v) {
    v.h.y = 0.f;
    v.l.y = 0.f;
    return v;
}

}  // namespace quapi
