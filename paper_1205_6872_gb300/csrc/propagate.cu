// Tensor-propagator kernels: the fused steady-state step with optional fused
// rho readout, the growth step, and the deterministic final rho reduction.
//
// Step (Sec. I: multiply the augmented tensor A by the propagator tensor T and
// sum over the oldest path index; T is never stored, it is rebuilt from small
// factor tables):
//   input  A_in[f * M2 + old]       f = the newer n_in-1 path points, old = the oldest
//   output A_out[x * F + f] = hi[x][f_hi] * lo[x][f_lo] * sum_old isum[x][old] * A_in[f*M2 + old]
// with F = (M^2)^(n_in-1) and f = f_hi * lo_size + f_lo.  For the diagonal new
// points x = (s, s) every influence factor is exactly 1 (d(x) = 0), so those
// rows share the plain sum over old and only carry K (in hi).
//
// Readout (Sec. IV, allPoints / justFinalPoint): rho(t_n)[x] is the same
// product with the end-point tables, summed over f instead of stored; each CTA
// writes its partial sums (FP64) and rho_reduce_kernel adds them in CTA order.
//
// Memory access: every thread owns FPT consecutive fibers (FP32: 2, so that its
// 2 outputs per row form one 16-byte store); a warp reads one contiguous span
// of A_in and writes M2 contiguous 512-byte runs of A_out.  Persistent grid
// (a multiple of the SM count), static tile order, streaming cache hints.
#include <cstdio>

#include "quapi_internal.h"

namespace quapi {

int num_sms();

namespace {

template <int FORM> struct FormT;
template <> struct FormT<QUAPI_FP64> {
    using Elem = double2;
    using Tab = double2;
    static constexpr int FPT = 1;
};
template <> struct FormT<QUAPI_FP32> {
    using Elem = float2;
    using Tab = ff2;
    static constexpr int FPT = 2;
};

template <int M> __device__ __forceinline__ constexpr bool is_diag(int x) { return (x / M) == (x % M); }

template <int M> struct Split {
    // f -> (f_hi, f_lo) for lo_size = M2^j
    __device__ __forceinline__ static void split(uint32_t f, uint32_t lo_size, int lo_shift, uint32_t& hi,
                                                 uint32_t& lo) {
        if (M == 2) {
            hi = f >> lo_shift;
            lo = f & (lo_size - 1u);
        } else {
            hi = f / lo_size;
            lo = f - hi * lo_size;
        }
    }
};

// ---- per-form arithmetic -------------------------------------------------------
__device__ __forceinline__ double2 tmul(const double2& T, double2 v) { return cmul(T, v); }
__device__ __forceinline__ float2 tmul(const ff2& T, float2 v) { return ffmul(T, v); }

__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }

// Loads the FPT fibers of this thread (valid[u] says whether fiber u exists).
template <int M2, int FORM>
__device__ __forceinline__ void load_fibers(const typename FormT<FORM>::Elem* __restrict__ A, int64_t f0,
                                            int64_t F, typename FormT<FORM>::Elem (&a)[FormT<FORM>::FPT][M2],
                                            bool (&valid)[FormT<FORM>::FPT]) {
    constexpr int FPT = FormT<FORM>::FPT;
    using Elem = typename FormT<FORM>::Elem;
    if constexpr (FORM == QUAPI_FP32) {
        if (f0 + 1 < F) {
            // 2 fibers = M2 * 16 bytes, 16-byte aligned because f0 is even
            const float4* p = reinterpret_cast<const float4*>(A + f0 * M2);
            float4 v[M2];
#pragma unroll
            for (int q = 0; q < M2; ++q) v[q] = __ldcs(p + q);
#pragma unroll
            for (int q = 0; q < M2; ++q) {
                int e0 = 2 * q, e1 = 2 * q + 1;
                a[e0 / M2][e0 % M2] = make_float2(v[q].x, v[q].y);
                a[e1 / M2][e1 % M2] = make_float2(v[q].z, v[q].w);
            }
            valid[0] = valid[1] = true;
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < FPT; ++u) {
        valid[u] = (f0 + u) < F;
#pragma unroll
        for (int q = 0; q < M2; ++q) {
            a[u][q] = valid[u] ? ld_stream(A + (f0 + u) * M2 + q) : Elem{};
        }
    }
}

template <int M, int FORM>
__device__ __forceinline__ void store_row(typename FormT<FORM>::Elem* __restrict__ out, int64_t idx,
                                          const typename FormT<FORM>::Elem (&v)[FormT<FORM>::FPT],
                                          const bool (&valid)[FormT<FORM>::FPT]) {
    constexpr int FPT = FormT<FORM>::FPT;
    if constexpr (FORM == QUAPI_FP32 && M == 2) {
        if (valid[1]) {  // idx even (F even whenever 2 fibers exist)
            __stcs(reinterpret_cast<float4*>(out + idx), make_float4(v[0].x, v[0].y, v[1].x, v[1].y));
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < FPT; ++u)
        if (valid[u]) __stcs(out + idx + u, v[u]);
}

// Readout accumulators: FP64 form in double, FP32 form compensated in float.
template <int FORM> struct RhoAcc;
template <> struct RhoAcc<QUAPI_FP64> {
    double2 s;
    __device__ __forceinline__ void init() { s = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void add(double2 v) { s = cadd(s, v); }
    __device__ __forceinline__ double2 value() const { return s; }
};
template <> struct RhoAcc<QUAPI_FP32> {
    cacc32 a;
    __device__ __forceinline__ void init() { a.init(make_float2(0.f, 0.f)); }
    __device__ __forceinline__ void add(float2 v) { a.add(v); }
    __device__ __forceinline__ double2 value() const {
        return make_double2((double)a.s.x + (double)a.c.x, (double)a.s.y + (double)a.c.y);
    }
};

// Sum over the oldest index with the summed-digit table (compensated in FP32).
template <int M2>
__device__ __forceinline__ double2 row_sum(const double2* __restrict__ isum_row, const double2 (&a)[M2]) {
    double2 s = cmul(isum_row[0], a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cfma(isum_row[q], a[q], s);
    return s;
}
template <int M2>
__device__ __forceinline__ cacc32 row_sum(const ff2* __restrict__ isum_row, const float2 (&a)[M2]) {
    cacc32 acc;
    acc.init(ffmul(isum_row[0], a[0]));
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add(ffmul(isum_row[q], a[q]));
    return acc;
}
template <int M2> __device__ __forceinline__ double2 plain_sum(const double2 (&a)[M2]) {
    double2 s = a[0];
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cadd(s, a[q]);
    return s;
}
template <int M2> __device__ __forceinline__ cacc32 plain_sum(const float2 (&a)[M2]) {
    cacc32 acc;
    acc.init(a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add(a[q]);
    return acc;
}

// hi * (lo * S)
__device__ __forceinline__ double2 apply_p(const double2& hi, const double2& lo, double2 S) {
    return cmul(hi, cmul(lo, S));
}
__device__ __forceinline__ float2 apply_p(const ff2& hi, const ff2& lo, const cacc32& S) {
    return ffmul(hi, ffmul2(lo, S.s, S.c));
}
__device__ __forceinline__ double2 apply_hi(const double2& hi, double2 S) { return cmul(hi, S); }
__device__ __forceinline__ float2 apply_hi(const ff2& hi, const cacc32& S) { return ffmul2(hi, S.s, S.c); }

template <int M, int FORM, bool WRITE, bool READ, bool DIAG>
__global__ void __launch_bounds__(kThreads) step_kernel(StepArgs args) {
    constexpr int M2 = M * M;
    using F_ = FormT<FORM>;
    using Elem = typename F_::Elem;
    using Tab = typename F_::Tab;
    constexpr int FPT = F_::FPT;
    constexpr int TILE = kThreads * FPT;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tab* s_isum = reinterpret_cast<Tab*>(smem_raw);
    Tab* s_isume = s_isum + M2 * M2;
    Tab* s_lo = s_isume + M2 * M2;
    Tab* s_loe = s_lo + M2 * args.lo_size;

    const Tab* g_isum = reinterpret_cast<const Tab*>(args.isum);
    const Tab* g_lo = reinterpret_cast<const Tab*>(args.lo);
    const Tab* g_hi = reinterpret_cast<const Tab*>(args.hi);
    const Tab* g_isume = reinterpret_cast<const Tab*>(args.isum_e);
    const Tab* g_loe = reinterpret_cast<const Tab*>(args.lo_e);
    const Tab* g_hie = reinterpret_cast<const Tab*>(args.hi_e);
    const uint32_t lo_size = (uint32_t)args.lo_size;
    const int64_t hi_size = args.F / args.lo_size;

    for (int e = threadIdx.x; e < M2 * M2; e += kThreads) {
        if (WRITE) s_isum[e] = g_isum[e];
        if (READ) s_isume[e] = g_isume[e];
    }
    for (int e = threadIdx.x; e < M2 * (int)lo_size; e += kThreads) {
        if (WRITE) s_lo[e] = g_lo[e];
        if (READ) s_loe[e] = g_loe[e];
    }
    __syncthreads();

    RhoAcc<FORM> racc[M2];
    if (READ) {
#pragma unroll
        for (int x = 0; x < M2; ++x) racc[x].init();
    }

    const Elem* __restrict__ A = reinterpret_cast<const Elem*>(args.A_in);
    Elem* __restrict__ out = reinterpret_cast<Elem*>(args.A_out);
    const int64_t F = args.F;
    const int64_t ntiles = (F + TILE - 1) / TILE;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t f0 = tile * TILE + (int64_t)threadIdx.x * FPT;
        Elem a[FPT][M2];
        bool valid[FPT];
        load_fibers<M2, FORM>(A, f0, F, a, valid);
        if (!valid[0]) continue;

        uint32_t fhi[FPT], flo[FPT];
#pragma unroll
        for (int u = 0; u < FPT; ++u) Split<M>::split((uint32_t)(f0 + u), lo_size, args.lo_shift, fhi[u], flo[u]);

        // diagonal rows: shared plain sum, only K (in hi) applies
        decltype(plain_sum<M2>(a[0])) Sd[FPT];
        if (DIAG) {
#pragma unroll
            for (int u = 0; u < FPT; ++u) Sd[u] = plain_sum<M2>(a[u]);
        }
#pragma unroll
        for (int x = 0; x < M2; ++x) {
            Elem vout[FPT];
            Elem vread[FPT];
            const bool diag_row = DIAG && is_diag<M>(x);
#pragma unroll
            for (int u = 0; u < FPT; ++u) {
                if (!valid[u]) {
                    vout[u] = Elem{};
                    vread[u] = Elem{};
                    continue;
                }
                if (diag_row) {
                    const int64_t hidx = (int64_t)x * hi_size + fhi[u];
                    if (WRITE) {
                        vout[u] = apply_hi(g_hi[hidx], Sd[u]);
                        vread[u] = vout[u];
                    } else {
                        vread[u] = apply_hi(g_hie[hidx], Sd[u]);
                    }
                } else {
                    if (WRITE) {
                        auto S = row_sum<M2>(s_isum + x * M2, a[u]);
                        vout[u] = apply_p(g_hi[(int64_t)x * hi_size + fhi[u]], s_lo[x * lo_size + flo[u]], S);
                    }
                    if (READ) {
                        auto Se = row_sum<M2>(s_isume + x * M2, a[u]);
                        vread[u] = apply_p(g_hie[(int64_t)x * hi_size + fhi[u]], s_loe[x * lo_size + flo[u]], Se);
                    }
                }
                if (READ) racc[x].add(vread[u]);
            }
            if (WRITE) store_row<M, FORM>(out, (int64_t)x * F + f0, vout, valid);
        }
    }

    if (READ) {
        __shared__ double2 red[kThreads / 32][M2];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int x = 0; x < M2; ++x) {
            double2 v = racc[x].value();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, off);
                v.y += __shfl_down_sync(0xffffffffu, v.y, off);
            }
            if (lane == 0) red[warp][x] = v;
        }
        __syncthreads();
        if (threadIdx.x < M2) {
            double2 v = make_double2(0.0, 0.0);
            for (int w = 0; w < kThreads / 32; ++w) v = cadd(v, red[w][threadIdx.x]);
            args.partial[(int64_t)blockIdx.x * M2 + threadIdx.x] = v;
        }
    }
}

template <int M, int FORM>
__global__ void __launch_bounds__(kThreads) grow_kernel(const void* __restrict__ A_in_, void* __restrict__ A_out_,
                                                        int64_t S, const void* __restrict__ lo_,
                                                        const void* __restrict__ hi_, int64_t lo_size_,
                                                        int lo_shift) {
    constexpr int M2 = M * M;
    using Elem = typename FormT<FORM>::Elem;
    using Tab = typename FormT<FORM>::Tab;
    const Elem* A = reinterpret_cast<const Elem*>(A_in_);
    Elem* out = reinterpret_cast<Elem*>(A_out_);
    const Tab* lo = reinterpret_cast<const Tab*>(lo_);
    const Tab* hi = reinterpret_cast<const Tab*>(hi_);
    const uint32_t lo_size = (uint32_t)lo_size_;
    const int64_t hi_size = S / lo_size_;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        Elem v = A[i];
        uint32_t ih, il;
        Split<M>::split((uint32_t)i, lo_size, lo_shift, ih, il);
#pragma unroll
        for (int x = 0; x < M2; ++x) {
            Elem z = tmul(lo[(int64_t)x * lo_size + il], v);
            out[(int64_t)x * S + i] = tmul(hi[(int64_t)x * hi_size + ih], z);
        }
    }
}

__global__ void rho_reduce_kernel(const double2* __restrict__ partial, int nparts, int M2,
                                  double2* __restrict__ rho_out) {
    int x = threadIdx.x;
    if (x >= M2) return;
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < nparts; ++b) v = cadd(v, partial[(int64_t)b * M2 + x]);
    rho_out[x] = v;
}

template <int M, int FORM, bool W, bool R, bool D>
cudaError_t launch_variant(StepArgs& a, cudaStream_t st) {
    using Tab = typename FormT<FORM>::Tab;
    constexpr int M2 = M * M;
    constexpr int FPT = FormT<FORM>::FPT;
    size_t smem = sizeof(Tab) * (2 * M2 * M2 + 2 * M2 * (size_t)a.lo_size);
    auto kern = step_kernel<M, FORM, W, R, D>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // persistent grid: every resident CTA slot of every SM, capped by the tile count
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int64_t ntiles = (a.F + (int64_t)kThreads * FPT - 1) / ((int64_t)kThreads * FPT);
    int64_t g = (int64_t)num_sms() * occ;
    if (g > ntiles) g = ntiles;
    if (g > a.grid) g = a.grid;  // caller's cap (size of the partial-sum buffer)
    if (g < 1) g = 1;
    a.grid = (int)g;
    kern<<<a.grid, kThreads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int M, int FORM>
cudaError_t launch_step_mf(StepArgs& a, cudaStream_t st) {
    const bool W = a.A_out != nullptr, R = a.partial != nullptr;
    if (a.diag_fast) {
        if (W && R) return launch_variant<M, FORM, true, true, true>(a, st);
        if (W) return launch_variant<M, FORM, true, false, true>(a, st);
        if (R) return launch_variant<M, FORM, false, true, true>(a, st);
    } else {
        if (W && R) return launch_variant<M, FORM, true, true, false>(a, st);
        if (W) return launch_variant<M, FORM, true, false, false>(a, st);
        if (R) return launch_variant<M, FORM, false, true, false>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 1;
    }
    return sms;
}

cudaError_t launch_step(int M, int form, StepArgs& a, cudaStream_t st) {
    if (M == 2 && form == QUAPI_FP64) return launch_step_mf<2, QUAPI_FP64>(a, st);
    if (M == 2 && form == QUAPI_FP32) return launch_step_mf<2, QUAPI_FP32>(a, st);
    if (M == 3 && form == QUAPI_FP64) return launch_step_mf<3, QUAPI_FP64>(a, st);
    if (M == 3 && form == QUAPI_FP32) return launch_step_mf<3, QUAPI_FP32>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_grow(int M, int form, const void* A_in, void* A_out, int64_t S, const void* lo,
                        const void* hi, int64_t lo_size, int lo_shift, cudaStream_t st) {
    int64_t blocks = (S + kThreads - 1) / kThreads;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    if (blocks < 1) blocks = 1;
#define QUAPI_GROW(MM, FF) grow_kernel<MM, FF><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, S, lo, hi, lo_size, lo_shift)
    if (M == 2 && form == QUAPI_FP64) QUAPI_GROW(2, QUAPI_FP64);
    else if (M == 2 && form == QUAPI_FP32) QUAPI_GROW(2, QUAPI_FP32);
    else if (M == 3 && form == QUAPI_FP64) QUAPI_GROW(3, QUAPI_FP64);
    else if (M == 3 && form == QUAPI_FP32) QUAPI_GROW(3, QUAPI_FP32);
    else return cudaErrorInvalidValue;
#undef QUAPI_GROW
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rho_reduce(const double2* partial, int nparts, int M2, double2* rho_out, cudaStream_t st) {
    rho_reduce_kernel<<<1, 32, 0, st>>>(partial, nparts, M2, rho_out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace quapi
