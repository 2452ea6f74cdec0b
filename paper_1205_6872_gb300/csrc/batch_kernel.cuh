// The batched persistent kernel (device side), shared by the per-form translation units
// batch_fp64.cu, batch_fp32.cu and batch_df64.cu (compiled in parallel); the work list, plans,
// tuning and the C entry point live in batch.cu.  How the kernel works is described there.
#pragma once

#include <algorithm>
#include <cstdint>

#include "half_layout.cuh"
#include "step_math.cuh"

namespace quapi {
namespace batchk {

constexpr int kBThreads = 256;
constexpr int kResidentBytes = 32 * 1024;

struct BatchArgs {
    const BatchInst* inst;
    const int* resident;        // instance ids run whole in shared memory
    int nresident;
    const int* tiled;           // instance ids processed tile by tile
    int ntiled;
    int nwaves;                 // largest final step among the tiled instances
    const int64_t* wave_off;    // [nwaves + 2]: first item of wave n (wave 0 = resident items)
    const unsigned* need;       // [(nwaves + 1) x ntiled]: tiles instance k completes before step n
    const unsigned* ntiles;     // [(nwaves + 1) x ntiled]: tiles of instance k at step n (0: none)
    const uint4* items;         // [total_items - nresident]: (step n, tiled instance k, first tile, 0)
    int64_t total_items;
    unsigned long long* next_item;
    int* err;
    int group;
    uint64_t wait_ns;
};

// What one launch of the batched kernel needs (filled by the plan in batch.cu).
struct BatchLaunch {
    BatchArgs args{};
    int M = 0;
    int fpt = 0;
    bool half_only = false;  // every tiled instance in the half layout
    size_t smem = 0;         // dynamic shared memory of the resident kernel: the largest resident instance's tensors
    int grid = 0;            // tiled kernel; 0: sized from the occupancy at the first launch
    cudaStream_t side = nullptr;               // the resident kernel's stream
    cudaEvent_t fork = nullptr, join = nullptr;  // st -> side before it, side -> st after it
};

// Per-form launchers (one translation unit each).  prep = true: only set the kernel's
// shared-memory attribute and size the grid.
cudaError_t launch_batch_fp64(BatchLaunch& L, cudaStream_t st, bool prep);
cudaError_t launch_batch_fp32(BatchLaunch& L, cudaStream_t st, bool prep);
cudaError_t launch_batch_df64(BatchLaunch& L, cudaStream_t st, bool prep);

namespace {

using namespace math;

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int M, int FORM> __device__ __forceinline__ OpTabs<M, FORM> tabs_of(const OpRef& r) {
    using Tab = typename Form<FORM>::Tab;
    OpTabs<M, FORM> t;
    t.isum = reinterpret_cast<const Tab*>(r.isum);
    t.lo = reinterpret_cast<const Tab*>(r.lo);
    t.hi = reinterpret_cast<const Tab*>(r.hi);
    t.lo_size = (uint32_t)r.lo_size;
    t.lo_shift = r.lo_shift;
    t.hi_size = r.hi_size;
    return t;
}

template <int FORM> __device__ __forceinline__ typename Form<FORM>::Elem from_d(double2 v);
template <> __device__ __forceinline__ double2 from_d<QUAPI_FP64>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d<QUAPI_FP32>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}
template <> __device__ __forceinline__ df2 from_d<QUAPI_DF64>(double2 v) {  // hi = RN32(v), lo = RN32(v - hi)
    df2 r;
    r.h = make_float2((float)v.x, (float)v.y);
    r.l = make_float2((float)(v.x - (double)r.h.x), (float)(v.y - (double)r.h.y));
    return r;
}

__device__ __forceinline__ double2 ld_l2(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_l2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ df2 ld_l2(const df2* p) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    df2 r;
    r.h = make_float2(v.x, v.y);
    r.l = make_float2(v.z, v.w);
    return r;
}

__device__ double2 initial_entry(const BatchInst& I, int M, int x, const double2* rho0) {
    const double sp = I.s[x / M], sm = I.s[x % M], d = sp - sm;
    const double2 e = I.eta[I.self0_idx];
    const double re = -d * (e.x * sp - e.x * sm), im = -d * (e.y * sp + e.y * sm);
    double sn, cs;
    sincos(im, &sn, &cs);
    const double m = exp(re);
    return cmul(rho0[x], make_double2(m * cs, m * sn));
}

// Readout accumulator per row: FP64 plain, FP32 TwoSum-compensated.
template <int FORM> struct Acc;
template <> struct Acc<QUAPI_FP64> {
    double2 s;
    __device__ void init() { s = make_double2(0.0, 0.0); }
    __device__ void add(double2 v) { s = cadd(s, v); }
    __device__ double2 value() const { return s; }
};
template <> struct Acc<QUAPI_FP32> {
    cacc32 a;
    __device__ void init() { a.init(make_float2(0.f, 0.f)); }
    __device__ void add(float2 v) { a.add(v); }
    __device__ double2 value() const { return make_double2((double)a.s.x + a.c.x, (double)a.s.y + a.c.y); }
};
template <> struct Acc<QUAPI_DF64> {
    df2 a;
    __device__ void init() { a.h = a.l = make_float2(0.f, 0.f); }
    __device__ void add(const df2& v) { a = dfadd(a, v); }
    __device__ double2 value() const {
        return make_double2((double)a.h.x + (double)a.l.x, (double)a.h.y + (double)a.l.y);
    }
};

// Block-wide sum of acc (one value per row) in a fixed order; the result is
// valid in threads 0..M2-1 (thread x holds row x).
template <int M2, int FORM>
__device__ double2 block_rows_sum(const Acc<FORM> (&acc)[M2], double2 (*red)[M2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int x = 0; x < M2; ++x) {
        double2 v = acc[x].value();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, off);
            v.y += __shfl_down_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) red[warp][x] = v;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x < M2)
        for (int w = 0; w < kBThreads / 32; ++w) r = cadd(r, red[w][threadIdx.x]);
    __syncthreads();
    return r;
}

template <int M, int FORM>
__device__ void step_fiber_dispatch(const OpRef& op, const typename Form<FORM>::Elem (&a)[M * M], uint32_t f,
                                    typename Form<FORM>::Elem (&o)[M * M]) {
    const OpTabs<M, FORM> T = tabs_of<M, FORM>(op);
    if (op.diag)
        fiber_step<M, FORM, true>(T, a, f, o);
    else
        fiber_step<M, FORM, false>(T, a, f, o);
}

// ---- Hermitian half layout (M = 2) for tiled instances ----------------------------
// Positions, rows and conjugate partners as in the single-instance half-layout kernels: one
// canonical prefix gives rows 1, 0 and 3 of its fiber and row 1 of its conjugate prefix.

template <int FORM> __device__ __forceinline__ void ld_fiber4(const typename Form<FORM>::Elem* A, uint32_t c,
                                                             typename Form<FORM>::Elem (&a)[4]) {
    if constexpr (FORM == QUAPI_FP32) {
        const float4* p = reinterpret_cast<const float4*>(A + 4ull * c);
        const float4 v0 = __ldcg(p), v1 = __ldcg(p + 1);
        a[0] = make_float2(v0.x, v0.y);
        a[1] = make_float2(v0.z, v0.w);
        a[2] = make_float2(v1.x, v1.y);
        a[3] = make_float2(v1.z, v1.w);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = ld_l2(A + 4ull * c + q);
    }
}

// rows 0, 1, 3 of fiber a at prefix f (ONLY1: row 1 alone); the diagonal rows use the plain sum when
// the operation allows it
template <int FORM, bool ONLY1>
__device__ __forceinline__ void herm_rows_b(const OpTabs<2, FORM>& T, bool diag,
                                            const typename Form<FORM>::Elem (&a)[4], uint32_t f,
                                            typename Form<FORM>::Elem (&o)[4]) {
    using Elem = typename Form<FORM>::Elem;
    uint32_t fh, fl;
    T.split(f, fh, fl);
    if (!ONLY1) {
        if (diag) {
            Elem c;
            const Elem s = plain_dot<4>(a, c);
            o[0] = tab_mul2(ldt(T.hi + fh), s, c);
            o[3] = tab_mul2(ldt(T.hi + 3 * T.hi_size + fh), s, c);
        } else {
#pragma unroll
            for (int x = 0; x < 4; x += 3) {
                Elem c;
                const Elem s = tab_dot<4>(T.isum + x * 4, a, c);
                o[x] = tab_mul(ldt(T.hi + (int64_t)x * T.hi_size + fh), tab_mul2(ldt(T.lo + x * T.lo_size + fl), s, c));
            }
        }
    }
    Elem c;
    const Elem s = tab_dot<4>(T.isum + 4, a, c);
    o[1] = tab_mul(ldt(T.hi + T.hi_size + fh), tab_mul2(ldt(T.lo + T.lo_size + fl), s, c));
}

// Steady step over the tile's positions [tile_base, tile_base + kBThreads * FPT): warp w takes the
// 32 * FPT consecutive positions from tile_base + w * 32 * FPT, lane l the positions l, l + 32, ...
// of that chunk.  A chunk inside one digit-1 block of level >= 2 is decoded once per warp (its
// prefixes are then consecutive plain indices f = f0 + i with fiber positions h0 + i / 4);
// otherwise each position is decoded on its own.
template <int FORM, int FPT>
__device__ void herm_step_tile(const OpRef& op, const void* in, void* outv, int np, int64_t tile_base) {
    using Elem = typename Form<FORM>::Elem;
    constexpr int remap[4] = {0, 2, 1, 3};
    constexpr uint32_t kWarpChunk = 32u * FPT;
    const OpTabs<2, FORM> T = tabs_of<2, FORM>(op);
    const Elem* A = reinterpret_cast<const Elem*>(in);
    Elem* out = reinterpret_cast<Elem*>(outv);
    const uint32_t npre = half_count32(np);
    const uint32_t top = (np >= 1) ? (1u << (2 * (np - 1))) : 0u;
    const uint32_t cnh = (np >= 1) ? half_count32(np - 1) : 0u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t cb = (uint32_t)tile_base + (threadIdx.x >> 5) * kWarpChunk;
    if (cb >= npre) return;
    uint32_t f0, h0;
    bool sc0, shc0;
    half_decode_pair(cb, np, f0, sc0, h0, shc0);
    const uint32_t t = (f0 ^ (f0 >> 1)) & 0x55555555u;
    const uint32_t r1 = t ? (1u << (31 - __clz(t))) : 0u;
    const bool fast = !sc0 && !shc0 && (f0 & 3u) == 0u && (f0 & (r1 - 1u)) + kWarpChunk <= r1;
#pragma unroll 1
    for (uint32_t i = lane; i < kWarpChunk; i += 32) {
        const uint32_t c = cb + i;
        if (c >= npre) break;
        uint32_t f, h;
        bool sc, shc;
        if (fast) {
            f = f0 + i;
            h = h0 + (i >> 2);
            sc = false;
            shc = false;
        } else {
            half_decode_pair(c, np, f, sc, h, shc);
        }
        Elem a[4], o[4];
        ld_fiber4<FORM>(A, c, a);
        herm_rows_b<FORM, false>(T, op.diag != 0, a, f, o);
        if (np == 0) {
            out[0] = o[0];
            out[1] = o[1];
            out[2] = conjv(o[1]);
            out[3] = o[3];
            continue;
        }
        const uint32_t b0 = 4u * (top + h), b3 = 4u * (top + cnh + h), fl = f & 3u;
        out[f] = o[1];
        out[b0 + fl] = o[0];
        out[b3 + fl] = o[3];
        if (!sc) {
            Elem b[4], ob[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = conjv(a[remap[q]]);
            const uint32_t fb = conj_digits(f);
            herm_rows_b<FORM, true>(T, op.diag != 0, b, fb, ob);
            out[fb] = ob[1];
            if (shc) {
                out[b0 + 2] = conjv(o[0]);
                out[b3 + 2] = conjv(o[3]);
            }
        }
    }
}

// Readout contributions of positions c = base + u * kBThreads + threadIdx.x (np-digit prefixes):
// row 1 over f and its conjugate, twice the real part of rows 0 and 3 (their partners are conjugates);
// row 2 of rho is the conjugate of row 1 and is filled in by the caller.
template <int FORM, int FPT>
__device__ void herm_read_tile(const OpRef& op, const void* in, int np, int64_t tile_base, Acc<FORM> (&acc)[4]) {
    using Elem = typename Form<FORM>::Elem;
    constexpr int remap[4] = {0, 2, 1, 3};
    const OpTabs<2, FORM> T = tabs_of<2, FORM>(op);
    const Elem* A = reinterpret_cast<const Elem*>(in);
    const uint32_t npre = half_count32(np);
#pragma unroll 1
    for (int u = 0; u < FPT; ++u) {
        const uint32_t c = (uint32_t)tile_base + u * kBThreads + threadIdx.x;
        if (c >= npre) break;
        uint32_t f;
        bool sc;
        half_decode(c, np, f, sc);
        Elem a[4], r[4];
        ld_fiber4<FORM>(A, c, a);
        herm_rows_b<FORM, false>(T, op.diag != 0, a, f, r);
        acc[1].add(r[1]);
        if (!sc) {
            Elem b[4], rb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = conjv(a[remap[q]]);
            herm_rows_b<FORM, true>(T, op.diag != 0, b, conj_digits(f), rb);
            acc[1].add(rb[1]);
            acc[0].add(twice_real(r[0]));
            acc[3].add(twice_real(r[3]));
        } else {
            acc[0].add(real_part(r[0]));
            acc[3].add(real_part(r[3]));
        }
    }
}

// Growth n_in -> n_in + 1 digits: stored input entries e = base + u * kBThreads + threadIdx.x.
template <int FORM, int FPT>
__device__ void herm_grow_tile(const OpRef& op, const void* in, void* outv, int n_in, int64_t tile_base) {
    using Elem = typename Form<FORM>::Elem;
    const OpTabs<2, FORM> T = tabs_of<2, FORM>(op);
    const Elem* A = reinterpret_cast<const Elem*>(in);
    Elem* out = reinterpret_cast<Elem*>(outv);
    const uint32_t S = 1u << (2 * n_in);          // plain row-1 block of the output
    const uint32_t Cp = half_count32(n_in - 1);  // canonical prefixes of the input
    auto Pm = [&](int x, uint32_t idx, Elem w) {
        uint32_t ih, il;
        T.split(idx, ih, il);
        return tab_mul(ldt(T.hi + (int64_t)x * T.hi_size + ih), tab_mul(ldt(T.lo + x * T.lo_size + il), w));
    };
#pragma unroll 1
    for (int u = 0; u < FPT; ++u) {
        const uint32_t e = (uint32_t)tile_base + u * kBThreads + threadIdx.x;
        if (e >= 4u * Cp) break;
        const uint32_t c = e >> 2, d = e & 3u;
        uint32_t P;
        bool scP;
        half_decode(c, n_in - 1, P, scP);
        const uint32_t i = (P << 2) | d;
        const Elem v = ld_l2(A + e);
        if (!(scP && d == 2u)) {  // (P, 2) of a self-conjugate P is written from (P, 1)
            out[i] = Pm(1, i, v);
            if (!(scP && (d == 0u || d == 3u))) {
                const uint32_t ib = conj_digits(i);
                out[ib] = Pm(1, ib, conjv(v));
            }
        }
        out[4u * ((S >> 2) + c) + d] = Pm(0, i, v);
        out[4u * ((S >> 2) + Cp + c) + d] = Pm(3, i, v);
    }
}

// ---- Hermitian half layout, M = 3, for tiled instances ------------------------------------
// Positions, rows and conjugate partners as in the single-instance M = 3 half-layout kernels: one
// canonical prefix f gives all nine rows of its fiber; rows 1, 2, 5 go to their plain blocks at f,
// rows 3, 6, 7 (conjugated) to the same blocks at conj f, rows 0, 4, 8 to the fiber of (x, f / 9).
// Each position of the tile is decoded on its own (base-9 walk).

template <int FORM, int FPT>
__device__ void herm3_step_tile(const OpRef& op, const void* in, void* outv, int np, int64_t tile_base) {
    using Elem = typename Form<FORM>::Elem;
    const Elem* A = reinterpret_cast<const Elem*>(in);
    Elem* out = reinterpret_cast<Elem*>(outv);
    const uint32_t npre = half3_count(np);
    const uint32_t P1 = pow9(np);
    const uint32_t sbase = (np >= 1) ? P1 / 3u : 0u;
    const uint32_t cnh = (np >= 1) ? half3_count(np - 1) : 0u;
#pragma unroll 1
    for (int u = 0; u < FPT; ++u) {
        const uint32_t c = (uint32_t)tile_base + u * kBThreads + threadIdx.x;
        if (c >= npre) break;
        uint32_t f, h;
        bool sc, shc;
        half3_decode_pair(c, np, f, sc, h, shc);
        Elem a[9], o[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) a[q] = ld_l2(A + 9ull * c + q);
        step_fiber_dispatch<3, FORM>(op, a, f, o);
        if (np == 0) {
#pragma unroll
            for (int x = 0; x < 9; ++x) out[x] = o[x];
            continue;
        }
        const uint32_t f0 = f % 9u, e0 = 9u * (sbase + h) + f0, e1 = e0 - f0 + conj3(f0);
        out[f] = o[1];
        out[P1 + f] = o[2];
        out[2u * P1 + f] = o[5];
        out[e0] = o[0];
        out[e0 + 9u * cnh] = o[4];
        out[e0 + 18u * cnh] = o[8];
        if (!sc) {
            const uint32_t fb = conj_digits3(f, np);
            out[fb] = conjv(o[3]);
            out[P1 + fb] = conjv(o[6]);
            out[2u * P1 + fb] = conjv(o[7]);
            if (shc) {  // the fiber of a self-conjugate (x, f / 9) keeps every last digit
                out[e1] = conjv(o[0]);
                out[e1 + 9u * cnh] = conjv(o[4]);
                out[e1 + 18u * cnh] = conjv(o[8]);
            }
        }
    }
}

// Readout contributions of positions c = base + u * kBThreads + threadIdx.x: rows 1, 2, 5 over f and its
// conjugate (r_x + conj r_conj(x)), twice the real part of rows 0, 4, 8; rows 3, 6, 7 of rho are the
// conjugates of rows 1, 2, 5 and are filled in by the caller.
template <int FORM, int FPT>
__device__ void herm3_read_tile(const OpRef& op, const void* in, int np, int64_t tile_base, Acc<FORM> (&acc)[9]) {
    using Elem = typename Form<FORM>::Elem;
    const Elem* A = reinterpret_cast<const Elem*>(in);
    const uint32_t npre = half3_count(np);
#pragma unroll 1
    for (int u = 0; u < FPT; ++u) {
        const uint32_t c = (uint32_t)tile_base + u * kBThreads + threadIdx.x;
        if (c >= npre) break;
        uint32_t f;
        bool sc;
        half3_decode(c, np, f, sc);
        Elem a[9], r[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) a[q] = ld_l2(A + 9ull * c + q);
        step_fiber_dispatch<3, FORM>(op, a, f, r);
        acc[1].add(r[1]);
        acc[2].add(r[2]);
        acc[5].add(r[5]);
        if (!sc) {
            acc[1].add(conjv(r[3]));
            acc[2].add(conjv(r[6]));
            acc[5].add(conjv(r[7]));
            acc[0].add(twice_real(r[0]));
            acc[4].add(twice_real(r[4]));
            acc[8].add(twice_real(r[8]));
        } else {
            acc[0].add(real_part(r[0]));
            acc[4].add(real_part(r[4]));
            acc[8].add(real_part(r[8]));
        }
    }
}

// Growth n_in -> n_in + 1 digits in the M = 3 half layout: stored input entries
// e = base + u * kBThreads + threadIdx.x (the rules of herm3_grow_kernel).
template <int FORM, int FPT>
__device__ void herm3_grow_tile(const OpRef& op, const void* in, void* outv, int n_in, int64_t tile_base) {
    using Elem = typename Form<FORM>::Elem;
    const OpTabs<3, FORM> T = tabs_of<3, FORM>(op);
    const Elem* A = reinterpret_cast<const Elem*>(in);
    Elem* out = reinterpret_cast<Elem*>(outv);
    const uint32_t S = pow9(n_in);
    const uint32_t Cp = half3_count(n_in - 1);
    const uint32_t sbase = S / 3u;
    auto Pm = [&](int x, uint32_t idx, Elem w) {
        uint32_t ih, il;
        T.split(idx, ih, il);
        return tab_mul(ldt(T.hi + (int64_t)x * T.hi_size + ih), tab_mul(ldt(T.lo + x * T.lo_size + il), w));
    };
#pragma unroll 1
    for (int u = 0; u < FPT; ++u) {
        const uint32_t e = (uint32_t)tile_base + u * kBThreads + threadIdx.x;
        if (e >= 9u * Cp) break;
        const uint32_t c = e / 9u, d = e % 9u;
        uint32_t P;
        bool scP;
        half3_decode(c, n_in - 1, P, scP);
        const uint32_t i = P * 9u + d;
        const Elem v = ld_l2(A + e);
        const bool dtop = (d == 1u || d == 2u || d == 5u);
        if (!(scP && !dtop && !self3(d))) {
            out[i] = Pm(1, i, v);
            out[S + i] = Pm(2, i, v);
            out[2u * S + i] = Pm(5, i, v);
        }
        if (!scP || dtop) {
            const uint32_t ib = conj_digits3(i, n_in);
            const Elem vb = conjv(v);
            out[ib] = Pm(1, ib, vb);
            out[S + ib] = Pm(2, ib, vb);
            out[2u * S + ib] = Pm(5, ib, vb);
        }
        out[9u * (sbase + c) + d] = Pm(0, i, v);
        out[9u * (sbase + Cp + c) + d] = Pm(4, i, v);
        out[9u * (sbase + 2u * Cp + c) + d] = Pm(8, i, v);
    }
}

// One instance, every step in shared memory (resident instances).
template <int M, int FORM>
__device__ void run_resident(const BatchInst& I, unsigned char* smem, double2 (*red)[M * M]) {
    constexpr int M2 = M * M;
    using Elem = typename Form<FORM>::Elem;
    int64_t cap = 1;
    for (int i = 0; i < I.L; ++i) cap *= M2;
    Elem* bufA = reinterpret_cast<Elem*>(smem);
    Elem* bufB = bufA + cap;
    if (threadIdx.x < M2) bufA[threadIdx.x] = from_d<FORM>(initial_entry(I, M, threadIdx.x, I.rho0));
    __syncthreads();
    for (int n = 1; n < I.N; ++n) {
        if (n < I.L) {
            const OpTabs<M, FORM> T = tabs_of<M, FORM>(I.grow[n]);
            int64_t S = 1;
            for (int i = 0; i < n; ++i) S *= M2;
            for (int64_t i = threadIdx.x; i < S; i += kBThreads) {
                Elem o[M2];
                entry_grow<M, FORM>(T, bufA[i], (uint32_t)i, o);
#pragma unroll
                for (int x = 0; x < M2; ++x) bufB[x * S + i] = o[x];
            }
        } else {
            const OpRef& op = (n == I.L) ? I.step_first : I.step;
            const int64_t F = cap / M2;
            for (int64_t f = threadIdx.x; f < F; f += kBThreads) {
                Elem a[M2], o[M2];
#pragma unroll
                for (int q = 0; q < M2; ++q) a[q] = bufA[f * M2 + q];
                step_fiber_dispatch<M, FORM>(op, a, (uint32_t)f, o);
#pragma unroll
                for (int x = 0; x < M2; ++x) bufB[x * F + f] = o[x];
            }
        }
        __syncthreads();
        Elem* t = bufA;
        bufA = bufB;
        bufB = t;
    }
    // readout of rho(t_N) from A_{N-1}
    int64_t Fr = 1;
    for (int i = 1; i < I.read.n_in; ++i) Fr *= M2;
    Acc<FORM> acc[M2];
#pragma unroll
    for (int x = 0; x < M2; ++x) acc[x].init();
    for (int64_t f = threadIdx.x; f < Fr; f += kBThreads) {
        Elem a[M2], o[M2];
#pragma unroll
        for (int q = 0; q < M2; ++q) a[q] = bufA[f * M2 + q];
        step_fiber_dispatch<M, FORM>(I.read, a, (uint32_t)f, o);
#pragma unroll
        for (int x = 0; x < M2; ++x) acc[x].add(o[x]);
    }
    const double2 r = block_rows_sum<M2, FORM>(acc, red);
    if (threadIdx.x < M2) I.rho_out[threadIdx.x] = r;
    __syncthreads();
}

// The shared-memory resident instances: one CTA per instance runs all of its steps (a kernel of its
// own, on a side branch of the captured graph, so that its shared memory and registers stay out of
// the tiled kernel).
template <int M, int FORM>
__global__ void __launch_bounds__(kBThreads) batch_resident_kernel(BatchArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double2 red[kBThreads / 32][M * M];
    for (int r = blockIdx.x; r < args.nresident; r += gridDim.x) run_resident<M, FORM>(args.inst[args.resident[r]], smem, red);
}

// Minimum resident CTAs per SM of the tiled kernel (a register cap).  HO: every tiled instance of the
// batch is in the Hermitian half layout (M = 2) and the full-layout tile code is left out.
template <int M, int FORM, bool HO> constexpr int batch_min_ctas() {
    if (FORM == QUAPI_DF64) return 2;
    if (HO) return 4;
    return M == 2 ? 3 : 1;
}

template <int M, int FORM, int FPT, bool HO>
__global__ void __launch_bounds__(kBThreads, batch_min_ctas<M, FORM, HO>()) batch_kernel(BatchArgs args) {
    constexpr int M2 = M * M;
    using Elem = typename Form<FORM>::Elem;
    constexpr int TE = kBThreads * FPT;  // fibers (or growth entries) per tile
    __shared__ long long s_item;
    __shared__ int s_stop;
    __shared__ double2 red[kBThreads / 32][M2];

    // the next item's number is taken while the current one runs (thread 0, after its dependency wait)
    if (threadIdx.x == 0) {
        const int e = *reinterpret_cast<volatile int*>(args.err);
        s_item = e ? -1LL : (long long)atomicAdd(args.next_item, 1ull);
    }
    __syncthreads();
    for (;;) {
        const long long g = s_item;
        __syncthreads();  // every thread holds g before thread 0 writes the next number
        if (g < 0 || g >= args.total_items) break;
        const uint4 d = args.items[g];
        const int n = (int)d.x, k = (int)d.y;
        const unsigned nt = args.ntiles[(int64_t)n * args.ntiled + k];
        const unsigned t0 = d.z;
        const unsigned t1 = min(t0 + (unsigned)args.group, nt);
        const BatchInst& I = args.inst[args.tiled[k]];

        // every tile of the previous step of this instance must be complete
        if (threadIdx.x == 0) {
            const unsigned want = args.need[(int64_t)n * args.ntiled + k];
            volatile unsigned* d = I.done;
            int stop = 0;
            if (*d < want) {
                const uint64_t t_start = now_ns();
                while (*d < want) {
                    if (*reinterpret_cast<volatile int*>(args.err)) {
                        stop = 1;
                        break;
                    }
                    if (now_ns() - t_start > args.wait_ns) {
                        atomicExch(args.err, 1);
                        stop = 1;
                        break;
                    }
                }
            }
            __threadfence();
            s_stop = stop;
            const int e = *reinterpret_cast<volatile int*>(args.err);
            s_item = (stop || e) ? -1LL : (long long)atomicAdd(args.next_item, 1ull);
        }
        __syncthreads();
        if (s_stop) break;

        const void* in = I.buf[(n - 1) & 1];
        void* outv = I.buf[n & 1];
        for (unsigned t = t0; t < t1; ++t) {
            const int64_t base = (int64_t)t * TE + (int64_t)threadIdx.x * FPT;
            const bool herm = HO || I.herm;
            if (herm && n < I.N) {
                if constexpr (M == 2) {
                    if (n < I.L) herm_grow_tile<FORM, FPT>(I.grow[n], in, outv, n, (int64_t)t * TE);
                    else herm_step_tile<FORM, FPT>(n == I.L ? I.step_first : I.step, in, outv, I.L - 1, (int64_t)t * TE);
                } else if constexpr (!HO) {
                    if (n < I.L) herm3_grow_tile<FORM, FPT>(I.grow[n], in, outv, n, (int64_t)t * TE);
                    else herm3_step_tile<FORM, FPT>(n == I.L ? I.step_first : I.step, in, outv, I.L - 1, (int64_t)t * TE);
                }
            } else if (!HO && n < I.L && n < I.N) {
                int64_t S = 1;
                for (int i = 0; i < n; ++i) S *= M2;
                const OpTabs<M, FORM> T = tabs_of<M, FORM>(I.grow[n]);
                const Elem* A = reinterpret_cast<const Elem*>(in);
                Elem* out = reinterpret_cast<Elem*>(outv);
#pragma unroll
                for (int u = 0; u < FPT; ++u) {
                    const int64_t i = base + u;
                    if (i < S) {
                        Elem o[M2];
                        entry_grow<M, FORM>(T, ld_l2(A + i), (uint32_t)i, o);
#pragma unroll
                        for (int x = 0; x < M2; ++x) out[x * S + i] = o[x];
                    }
                }
            } else if (!HO && n < I.N) {
                int64_t F = 1;
                for (int i = 1; i < I.L; ++i) F *= M2;
                const OpRef& op = (n == I.L) ? I.step_first : I.step;
                const Elem* A = reinterpret_cast<const Elem*>(in);
                Elem* out = reinterpret_cast<Elem*>(outv);
                if constexpr (M == 2 && FORM == QUAPI_FP32 && FPT % 2 == 0) {
                    // pairs of fibers: 64-byte aligned loads, 16-byte stores per row (F is even here)
#pragma unroll
                    for (int u = 0; u < FPT; u += 2) {
                        const int64_t f = base + u;
                        if (f + 1 < F) {
                            const float4* p4 = reinterpret_cast<const float4*>(A + f * M2);
                            float4 v[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) v[q] = __ldcg(p4 + q);
                            Elem a0[M2] = {make_float2(v[0].x, v[0].y), make_float2(v[0].z, v[0].w),
                                           make_float2(v[1].x, v[1].y), make_float2(v[1].z, v[1].w)};
                            Elem a1[M2] = {make_float2(v[2].x, v[2].y), make_float2(v[2].z, v[2].w),
                                           make_float2(v[3].x, v[3].y), make_float2(v[3].z, v[3].w)};
                            Elem o0[M2], o1[M2];
                            step_fiber_dispatch<M, FORM>(op, a0, (uint32_t)f, o0);
                            step_fiber_dispatch<M, FORM>(op, a1, (uint32_t)(f + 1), o1);
#pragma unroll
                            for (int x = 0; x < M2; ++x)
                                __stcg(reinterpret_cast<float4*>(out + x * F + f),
                                       make_float4(o0[x].x, o0[x].y, o1[x].x, o1[x].y));
                        } else if (f < F) {
                            Elem a[M2], o[M2];
#pragma unroll
                            for (int q = 0; q < M2; ++q) a[q] = ld_l2(A + f * M2 + q);
                            step_fiber_dispatch<M, FORM>(op, a, (uint32_t)f, o);
#pragma unroll
                            for (int x = 0; x < M2; ++x) out[x * F + f] = o[x];
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < FPT; ++u) {
                        const int64_t f = base + u;
                        if (f < F) {
                            Elem a[M2], o[M2];
#pragma unroll
                            for (int q = 0; q < M2; ++q) a[q] = ld_l2(A + f * M2 + q);
                            step_fiber_dispatch<M, FORM>(op, a, (uint32_t)f, o);
#pragma unroll
                            for (int x = 0; x < M2; ++x) out[x * F + f] = o[x];
                        }
                    }
                }
            } else {
                int64_t F = 1;
                for (int i = 1; i < I.read.n_in; ++i) F *= M2;
                const Elem* A = reinterpret_cast<const Elem*>(in);
                Acc<FORM> acc[M2];
#pragma unroll
                for (int x = 0; x < M2; ++x) acc[x].init();
                if (herm) {
                    if constexpr (M == 2) herm_read_tile<FORM, FPT>(I.read, in, I.read.n_in - 1, (int64_t)t * TE, acc);
                    else if constexpr (!HO) herm3_read_tile<FORM, FPT>(I.read, in, I.read.n_in - 1, (int64_t)t * TE, acc);
                } else if constexpr (!HO) {
#pragma unroll
                    for (int u = 0; u < FPT; ++u) {
                        const int64_t f = base + u;
                        if (f < F) {
                            Elem a[M2], o[M2];
#pragma unroll
                            for (int q = 0; q < M2; ++q) a[q] = ld_l2(A + f * M2 + q);
                            step_fiber_dispatch<M, FORM>(I.read, a, (uint32_t)f, o);
#pragma unroll
                            for (int x = 0; x < M2; ++x) acc[x].add(o[x]);
                        }
                    }
                }
                const double2 v = block_rows_sum<M2, FORM>(acc, red);
                if (threadIdx.x < M2) {
                    // half layout: the rows (a, b) with a > b are the conjugates of the rows (b, a) (their
                    // threads hold empty sums)
                    const int x = threadIdx.x, xa = x / M, xb = x % M;
                    if (!(herm && xa > xb)) I.partial[(int64_t)t * M2 + x] = v;
                    if (herm && xa < xb) I.partial[(int64_t)t * M2 + xb * M + xa] = make_double2(v.x, -v.y);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    const unsigned prev = atomicAdd(I.read_done, 1u);
                    s_stop = (prev + 1 == nt) ? 2 : 0;
                    if (s_stop == 2) __threadfence();
                }
                __syncthreads();
                if (s_stop == 2 && threadIdx.x < M2) {
                    double2 sum = make_double2(0.0, 0.0);
                    for (unsigned p = 0; p < nt; ++p) sum = cadd(sum, __ldcg(I.partial + (int64_t)p * M2 + threadIdx.x));
                    I.rho_out[threadIdx.x] = sum;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(I.done, t1 - t0);
        }
    }
}

template <int M, int FORM>
__global__ void batch_init_kernel(const BatchInst* inst, const int* tiled, int ntiled) {
    const int k = blockIdx.x;
    if (k >= ntiled) return;
    const BatchInst& I = inst[tiled[k]];
    const int x = threadIdx.x;
    if (x < M * M) {
        using Elem = typename Form<FORM>::Elem;
        reinterpret_cast<Elem*>(I.buf[0])[x] = from_d<FORM>(initial_entry(I, M, x, I.rho0));
    }
}

// Resident instances on the side stream (forked from and joined back to st through the events), the
// tiled instances on st.
template <int M, int FORM, int FPT> cudaError_t launch_batch(BatchLaunch& P, cudaStream_t st, bool prepare_only) {
    auto kern = P.half_only ? batch_kernel<M, FORM, FPT, (M == 2)> : batch_kernel<M, FORM, FPT, false>;
    auto rkern = batch_resident_kernel<M, FORM>;
    cudaError_t e;
    if (P.smem > 0 && (e = cudaFuncSetAttribute(rkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem)) !=
                          cudaSuccess)
        return e;
    if (P.grid == 0) {
        int occ = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBThreads, 0);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        P.grid = std::max(1, sms * std::max(occ, 1));
    }
    if (prepare_only) return cudaSuccess;
    if (P.args.nresident) {
        if ((e = cudaEventRecord(P.fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(P.side, P.fork, 0)) != cudaSuccess) return e;
        rkern<<<P.args.nresident, kBThreads, P.smem, P.side>>>(P.args);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(P.join, P.side)) != cudaSuccess) return e;
    }
    if (P.args.ntiled) {
        batch_init_kernel<M, FORM><<<P.args.ntiled, 32, 0, st>>>(P.args.inst, P.args.tiled, P.args.ntiled);
        kern<<<P.grid, kBThreads, 0, st>>>(P.args);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (P.args.nresident && (e = cudaStreamWaitEvent(st, P.join, 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <int M, int FORM> cudaError_t launch_batch_fpt(BatchLaunch& P, cudaStream_t st, bool prep) {
    switch (P.fpt) {
        case 1: return launch_batch<M, FORM, 1>(P, st, prep);
        case 4: return launch_batch<M, FORM, 4>(P, st, prep);
        case 8:  // the plan only asks for 8 with M = 2 FP32 (its tiles are sized for the same FPT)
            if constexpr (M == 2 && FORM == QUAPI_FP32) return launch_batch<M, FORM, 8>(P, st, prep);
            return cudaErrorInvalidValue;
        default: return launch_batch<M, FORM, 2>(P, st, prep);
    }
}

template <int FORM> cudaError_t launch_batch_form(BatchLaunch& P, cudaStream_t st, bool prep) {
    if (P.M == 2) return launch_batch_fpt<2, FORM>(P, st, prep);
    if (P.M == 3) return launch_batch_fpt<3, FORM>(P, st, prep);
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace batchk
}  // namespace quapi
