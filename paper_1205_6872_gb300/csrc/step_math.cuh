// Per-entry arithmetic of one tensor operation, shared by the batched kernel.
//
// For the new path point x and a kept index i = i_hi * lo_size + i_lo:
//   growth:   out[x] = hi[x][i_hi] * lo[x][i_lo] * A[i]
//   step:     out[x] = hi[x][f_hi] * lo[x][f_lo] * sum_old isum[x][old] * A[f * M2 + old]
// (Sec. I, tensor propagator: T applied to A, then the sum over the oldest
// path index).  Diagonal new points x = (s, s) have d(x) = 0, so every
// influence factor is 1: their rows are the plain sum times hi (K only).
#pragma once

#include "quapi_internal.h"

namespace quapi {
namespace math {

template <int FORM> struct Form;
template <> struct Form<QUAPI_FP64> {
    using Elem = double2;
    using Tab = double2;
};
template <> struct Form<QUAPI_FP32> {
    using Elem = float2;
    using Tab = ff2;
};
template <> struct Form<QUAPI_DF64> {
    using Elem = df2;
    using Tab = tf2;
};

template <int M> __host__ __device__ constexpr bool diag_point(int x) { return (x / M) == (x % M); }

template <int M, int FORM> struct OpTabs {
    using Tab = typename Form<FORM>::Tab;
    const Tab* isum;
    const Tab* lo;
    const Tab* hi;
    uint32_t lo_size;
    int lo_shift;
    int64_t hi_size;

    __device__ __forceinline__ void split(uint32_t f, uint32_t& fh, uint32_t& fl) const {
        if (M == 2) {
            fh = f >> lo_shift;
            fl = f & (lo_size - 1u);
        } else {
            fh = f / lo_size;
            fl = f - fh * lo_size;
        }
    }
};

__device__ __forceinline__ double2 ldt(const double2* p) { return __ldg(p); }
__device__ __forceinline__ ff2 ldt(const ff2* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    ff2 t;
    t.hr = v.x;
    t.hi = v.y;
    t.lr = v.z;
    t.li = v.w;
    return t;
}

__device__ __forceinline__ tf2 ldt(const tf2* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    tf2 t;
    t.t1 = make_float2(a.x, a.y);
    t.t2 = make_float2(a.z, a.w);
    t.t3 = make_float2(b.x, b.y);
    t.pad = make_float2(0.f, 0.f);
    return t;
}

__device__ __forceinline__ double2 tab_mul(const double2& T, double2 v) { return cmul(T, v); }
__device__ __forceinline__ float2 tab_mul(const ff2& T, float2 v) { return ffmul(T, v); }
__device__ __forceinline__ df2 tab_mul(const tf2& T, const df2& v) { return tfmul(T, v); }

// sum_old isum[old] * a[old]: FP64 plain, FP32 Kahan-compensated (value = s + c)
template <int M2>
__device__ __forceinline__ double2 tab_dot(const double2* __restrict__ row, const double2 (&a)[M2], double2& c) {
    double2 s = cmul(ldt(row), a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cfma(ldt(row + q), a[q], s);
    c = make_double2(0.0, 0.0);
    return s;
}
template <int M2>
__device__ __forceinline__ float2 tab_dot(const ff2* __restrict__ row, const float2 (&a)[M2], float2& c) {
    kahan32 k;
    k.init(ffmul(ldt(row), a[0]));
#pragma unroll
    for (int q = 1; q < M2; ++q) k.add(ffmul(ldt(row + q), a[q]));
    c = k.c;
    return k.s;
}
// DF64: exact products added with TwoSum, renormalised once (c stays zero: the value is the pair)
template <int M2>
__device__ __forceinline__ df2 tab_dot(const tf2* __restrict__ row, const df2 (&a)[M2], df2& c) {
    dfacc acc;
    acc.init();
#pragma unroll
    for (int q = 0; q < M2; ++q) acc.add_prod(ldt(row + q), a[q]);
    c = df2{};
    return acc.value();
}
template <int M2> __device__ __forceinline__ df2 plain_dot(const df2 (&a)[M2], df2& c) {
    dfacc acc;
    acc.init();
#pragma unroll
    for (int q = 0; q < M2; ++q) acc.add_hl(a[q].h.x, a[q].l.x, a[q].h.y, a[q].l.y);
    c = df2{};
    return acc.value();
}
template <int M2> __device__ __forceinline__ double2 plain_dot(const double2 (&a)[M2], double2& c) {
    double2 s = a[0];
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cadd(s, a[q]);
    c = make_double2(0.0, 0.0);
    return s;
}
template <int M2> __device__ __forceinline__ float2 plain_dot(const float2 (&a)[M2], float2& c) {
    kahan32 k;
    k.init(a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) k.add(a[q]);
    c = k.c;
    return k.s;
}

// table * (s + c)
__device__ __forceinline__ double2 tab_mul2(const double2& T, double2 s, double2 /*c*/) { return cmul(T, s); }
__device__ __forceinline__ float2 tab_mul2(const ff2& T, float2 s, float2 c) { return ffmul2(T, s, c); }
__device__ __forceinline__ df2 tab_mul2(const tf2& T, const df2& s, const df2& /*c*/) { return tfmul(T, s); }

// All M2 outputs of fiber f (a = its M2 entries).  DIAG: diagonal rows use the
// plain sum and skip lo (valid when K sits in hi and isum has no K).
template <int M, int FORM, bool DIAG>
__device__ __forceinline__ void fiber_step(const OpTabs<M, FORM>& T,
                                           const typename Form<FORM>::Elem (&a)[M * M], uint32_t f,
                                           typename Form<FORM>::Elem (&out)[M * M]) {
    constexpr int M2 = M * M;
    using Elem = typename Form<FORM>::Elem;
    uint32_t fh, fl;
    T.split(f, fh, fl);
    Elem cd, sd;
    if (DIAG) sd = plain_dot<M2>(a, cd);
#pragma unroll
    for (int x = 0; x < M2; ++x) {
        const auto h = ldt(T.hi + (int64_t)x * T.hi_size + fh);
        if (DIAG && diag_point<M>(x)) {
            out[x] = tab_mul2(h, sd, cd);
        } else {
            Elem c;
            Elem s = tab_dot<M2>(T.isum + x * M2, a, c);
            out[x] = tab_mul(h, tab_mul2(ldt(T.lo + x * T.lo_size + fl), s, c));
        }
    }
}

// All M2 outputs of one growth input entry a = A[i].
template <int M, int FORM>
__device__ __forceinline__ void entry_grow(const OpTabs<M, FORM>& T, typename Form<FORM>::Elem a, uint32_t i,
                                           typename Form<FORM>::Elem (&out)[M * M]) {
    uint32_t ih, il;
    T.split(i, ih, il);
#pragma unroll
    for (int x = 0; x < M * M; ++x)
        out[x] = tab_mul(ldt(T.hi + (int64_t)x * T.hi_size + ih), tab_mul(ldt(T.lo + x * T.lo_size + il), a));
}

}  // namespace math
}  // namespace quapi
