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
// writes its partial sums (FP64) and rho_reduce_kernel adds them in a fixed order.
//
// Memory access: every thread owns FPT consecutive fibers (FP32 with M = 2: 2, so
// that its 2 outputs per row form one 16-byte store; otherwise 1); a warp reads one
// contiguous span of A_in and writes M2 contiguous runs of A_out.  Persistent grid
// (a multiple of the SM count), static tile order, streaming cache hints.  The
// M = 2 full layout normally takes the TMA-staged kernel; the Hermitian half
// layout has its own kernels (warp chunks of canonical positions, below).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>

#include "quapi_internal.h"
#include "half_layout.cuh"

namespace quapi {

int num_sms();

namespace {

// Programmatic dependent launch (the M = 2 half-layout step kernel): it lets the next kernel of its
// stream be scheduled while its own CTAs retire (pdl_allow_next), and waits for the previous kernel's
// completion and memory (pdl_wait) after staging its tables, before its first read of the tensor and
// before any global write.  Launched without the attribute, the wait returns at once.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class K>
cudaError_t launch_pdl(K kern, int grid, size_t smem, cudaStream_t st, const StepArgs& a, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int FORM> struct FormT;
template <> struct FormT<QUAPI_FP64> {
    using Elem = double2;
    using Tab = double2;
    static constexpr int FPT = 1;
    // FP64 is bound by its FP64 pipe: the folded table lo (x) isum saves one complex product per row
    static constexpr bool kFoldLo = true;
};
template <> struct FormT<QUAPI_FP32> {
    using Elem = float2;
    using Tab = ff2;
    static constexpr int FPT = 2;
    // bound by memory: lo and isum stay separate (both staged in shared memory)
    static constexpr bool kFoldLo = false;
};
template <> struct FormT<QUAPI_DF64> {
    using Elem = df2;
    using Tab = tf2;
    static constexpr int FPT = 1;
    static constexpr bool kFoldLo = false;
};

// Fibers per thread of the direct kernels: the form's count for M = 2; one for M = 3, whose
// 9-entry fibers would otherwise hold 2 x 9 inputs and outputs in registers (123 registers, 2 CTAs).
template <int M2, int FORM> __host__ __device__ constexpr int fibers_per_thread() {
    return M2 > 4 ? 1 : FormT<FORM>::FPT;
}

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

__device__ __forceinline__ df2 tmul(const tf2& T, df2 v) { return tfmul(T, v); }

__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ df2 ld_stream(const df2* p) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    df2 r;
    r.h = make_float2(v.x, v.y);
    r.l = make_float2(v.z, v.w);
    return r;
}
__device__ __forceinline__ void st_stream(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(df2* p, df2 v) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v.h.x, v.h.y, v.l.x, v.l.y));
}

// Loads the FPT fibers of this thread (valid[u] says whether fiber u exists).
template <int M2, int FORM>
__device__ __forceinline__ void load_fibers(const typename FormT<FORM>::Elem* __restrict__ A, int64_t f0,
                                            int64_t F,
                                            typename FormT<FORM>::Elem (&a)[fibers_per_thread<M2, FORM>()][M2],
                                            bool (&valid)[fibers_per_thread<M2, FORM>()]) {
    constexpr int FPT = fibers_per_thread<M2, FORM>();
    using Elem = typename FormT<FORM>::Elem;
    if constexpr (FORM == QUAPI_FP32 && FPT == 2) {
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
                                          const typename FormT<FORM>::Elem (&v)[fibers_per_thread<M * M, FORM>()],
                                          const bool (&valid)[fibers_per_thread<M * M, FORM>()]) {
    constexpr int FPT = fibers_per_thread<M * M, FORM>();
    if constexpr (FORM == QUAPI_FP32 && M == 2) {
        if (valid[1]) {  // idx even (F even whenever 2 fibers exist)
            __stcs(reinterpret_cast<float4*>(out + idx), make_float4(v[0].x, v[0].y, v[1].x, v[1].y));
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < FPT; ++u)
        if (valid[u]) st_stream(out + idx + u, v[u]);
}

// Readout accumulators: FP64 form in double, FP32 form compensated in float.
template <int FORM> struct RhoAcc;
template <> struct RhoAcc<QUAPI_FP64> {
    double2 s;
    __device__ __forceinline__ void init() { s = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void add(double2 v) { s = cadd(s, v); }
    __device__ __forceinline__ void add_re(double2 v, double k) { s.x += k * v.x; }  // + k Re(v)
    __device__ __forceinline__ double2 value() const { return s; }
};
template <> struct RhoAcc<QUAPI_FP32> {
    cacc32 a;
    __device__ __forceinline__ void init() { a.init(make_float2(0.f, 0.f)); }
    __device__ __forceinline__ void add(float2 v) { a.add(v); }
    __device__ __forceinline__ void add_re(float2 v, float k) { a.add_real(k * v.x); }  // k = 1 or 2: exact
    __device__ __forceinline__ double2 value() const {
        return make_double2((double)a.s.x + (double)a.c.x, (double)a.s.y + (double)a.c.y);
    }
};

template <> struct RhoAcc<QUAPI_DF64> {
    df2 a;
    __device__ __forceinline__ void init() { a.h = a.l = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(df2 v) { a = dfadd(a, v); }
    __device__ __forceinline__ void add_re(const df2& v, float k) {  // + k Re(v), k = 1 or 2 (exact scaling)
        float s, t;
        two_sum(a.h.x, k * v.h.x, s, t);
        t += a.l.x + k * v.l.x;
        fast_two_sum(s, t, a.h.x, a.l.x);
    }
    __device__ __forceinline__ double2 value() const {
        return make_double2((double)a.h.x + (double)a.l.x, (double)a.h.y + (double)a.l.y);
    }
};

// Sum over the oldest index with the summed-digit table.  FP32: Kahan-compensated, with FP32 products
// of the table's hi float when HIP (the fast path: no summed-index entry carries K), else products with
// both floats of the entry.  HIP changes nothing in the other forms.
template <int M2, bool HIP = false>
__device__ __forceinline__ double2 row_sum(const double2* __restrict__ isum_row, const double2 (&a)[M2]) {
    double2 s = cmul(isum_row[0], a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cfma(isum_row[q], a[q], s);
    return s;
}
template <int M2, bool HIP = false>
__device__ __forceinline__ kahan32 row_sum(const ff2* __restrict__ isum_row, const float2 (&a)[M2]) {
    kahan32 acc;
    acc.init(HIP ? fmul_hi(isum_row[0], a[0]) : ffmul(isum_row[0], a[0]));
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add(HIP ? fmul_hi(isum_row[q], a[q]) : ffmul(isum_row[q], a[q]));
    return acc;
}
template <int M2> __device__ __forceinline__ double2 plain_sum(const double2 (&a)[M2]) {
    double2 s = a[0];
#pragma unroll
    for (int q = 1; q < M2; ++q) s = cadd(s, a[q]);
    return s;
}
template <int M2> __device__ __forceinline__ kahan32 plain_sum(const float2 (&a)[M2]) {
    kahan32 acc;
    acc.init(a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add(a[q]);
    return acc;
}

// DF64 sums over the oldest index: started from the first term and left unrenormalised, because
// every caller multiplies them by a table entry next (the product takes the pair as it is)
template <int M2, bool HIP = false>
__device__ __forceinline__ df2 row_sum(const tf2* __restrict__ isum_row, const df2 (&a)[M2]) {
    dfacc acc;
    acc.init_prod(isum_row[0], a[0]);
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add_prod(isum_row[q], a[q]);
    return acc.raw();
}
template <int M2> __device__ __forceinline__ df2 plain_sum(const df2 (&a)[M2]) {
    dfacc acc;
    acc.init_hl(a[0].h.x, a[0].l.x, a[0].h.y, a[0].l.y);
#pragma unroll
    for (int q = 1; q < M2; ++q) acc.add_hl(a[q].h.x, a[q].l.x, a[q].h.y, a[q].l.y);
    return acc.raw();
}

// hi * (lo * S)
__device__ __forceinline__ float2 apply_p(const ff2& hi, const ff2& lo, const kahan32& S) {
    return ffmul(hi, ffmul2(lo, S.s, S.c));
}
__device__ __forceinline__ df2 apply_p(const tf2& hi, const tf2& lo, const df2& S) {
    return tfmul(hi, tfmul(lo, S));
}
__device__ __forceinline__ double2 apply_hi(const double2& hi, double2 S) { return cmul(hi, S); }
__device__ __forceinline__ df2 apply_hi(const tf2& hi, const df2& S) { return tfmul(hi, S); }
__device__ __forceinline__ float2 apply_hi(const ff2& hi, const kahan32& S) { return ffmul2(hi, S.s, S.c); }

// Folded row-1 table of the half-layout step (FP32 and DF64 forms, diagonal fast path).  With the
// fast path, rows 0 and 3 of the half layout carry only K (in hi), and row 1 (also the conjugate
// prefix's row 1) is hi[1][fh] * lo[1][fl] * sum_old isum[1][old] A[f, old].  The product
// lo[1][fl] isum[1][old] is formed once in FP64 at set-up (the w table, stored in the form's table
// format); the kernel stages its row 1 in shared memory with the summed index major, W1[old][fl], so
// that lanes with consecutive fl read consecutive entries (no bank conflicts), and the row costs one
// table product (hi) after the sum instead of two.
// The fast path needs at least one hi digit, so the lo table always resolves 4 digits there:
// lo_size = 256 is a compile-time stride (the launcher checks it).
constexpr uint32_t kFoldLo = 256;
template <int FORM> struct FoldRow {
    static constexpr size_t kEntryBytes = 0;
};
template <> struct FoldRow<QUAPI_FP32> {
    const ff2* w;  // [4][lo_size]
    static constexpr size_t kEntryBytes = sizeof(ff2);
    __device__ __forceinline__ ff2 at(int q, uint32_t fl) const { return w[q * kFoldLo + fl]; }
    __device__ __forceinline__ void stage(unsigned char* smem, const void* gw) {
        ff2* sw = reinterpret_cast<ff2*>(smem);
        const ff2* g = reinterpret_cast<const ff2*>(gw);
        for (uint32_t e = threadIdx.x; e < 4 * kFoldLo; e += kThreads) {
            const uint32_t q = e / kFoldLo, fl = e % kFoldLo;
            sw[e] = g[(kFoldLo + fl) * 4 + q];  // w[x = 1][fl][old = q]
        }
        w = sw;
    }
};
template <> struct FoldRow<QUAPI_DF64> {
    const float4* w12;  // [4][lo_size] {t1.re, t1.im, t2.re, t2.im}
    const float2* w3;   // [4][lo_size] t3
    static constexpr size_t kEntryBytes = sizeof(float4) + sizeof(float2);
    __device__ __forceinline__ tf2 at(int q, uint32_t fl) const {
        const float4 a = w12[q * kFoldLo + fl];
        tf2 t;
        t.t1 = make_float2(a.x, a.y);
        t.t2 = make_float2(a.z, a.w);
        t.t3 = w3[q * kFoldLo + fl];
        t.pad = make_float2(0.f, 0.f);
        return t;
    }
    __device__ __forceinline__ void stage(unsigned char* smem, const void* gw) {
        float4* s12 = reinterpret_cast<float4*>(smem);
        float2* s3 = reinterpret_cast<float2*>(smem + sizeof(float4) * 4 * kFoldLo);
        const tf2* g = reinterpret_cast<const tf2*>(gw);
        for (uint32_t e = threadIdx.x; e < 4 * kFoldLo; e += kThreads) {
            const uint32_t q = e / kFoldLo, fl = e % kFoldLo;
            const tf2 t = g[(kFoldLo + fl) * 4 + q];
            s12[e] = make_float4(t.t1.x, t.t1.y, t.t2.x, t.t2.y);
            s3[e] = t.t3;
        }
        w12 = s12;
        w3 = s3;
    }
};

// Forms whose half-layout fast path uses the folded row: DF64, which is bound by its FP32-pipe
// arithmetic (measured at memory length 14: 0.894 ms per step against 0.988 ms with lo and isum
// apart).  The FP32 step stays memory-bound and runs at a 32-register cap, where the fold's extra
// live state spills (0.376 ms against 0.370 ms); FP64 reads its own folded table through L1.
template <int FORM> __host__ __device__ constexpr bool herm_fold() { return FORM == QUAPI_DF64; }
// The other fast path that keeps lo and isum apart (FP32): rows 0 and 3 are diagonal there and row 2
// is written from the conjugate prefix's row 1, so only row 1 of both tables is staged (4 KB instead
// of 16 KB per CTA, which leaves more of the SM's L1 to the hi entries).
template <int FORM, bool DIAG> __host__ __device__ constexpr bool herm_row1() {
    return DIAG && !herm_fold<FORM>() && !FormT<FORM>::kFoldLo;
}

// sum_old W1[old][fl] * a[old] (fast path only): FP32 products of the hi float, Kahan-compensated;
// DF64 exact products added with TwoSum
__device__ __forceinline__ kahan32 fold_sum(const FoldRow<QUAPI_FP32>& W, uint32_t fl, const float2 (&a)[4]) {
    kahan32 acc;
    acc.init(fmul_hi(W.at(0, fl), a[0]));
#pragma unroll
    for (int q = 1; q < 4; ++q) acc.add(fmul_hi(W.at(q, fl), a[q]));
    return acc;
}
// DF64: left unrenormalised (it is multiplied by hi next)
__device__ __forceinline__ df2 fold_sum(const FoldRow<QUAPI_DF64>& W, uint32_t fl, const df2 (&a)[4]) {
    dfacc acc;
    acc.init_prod(W.at(0, fl), a[0]);
#pragma unroll
    for (int q = 1; q < 4; ++q) acc.add_prod(W.at(q, fl), a[q]);
    return acc.raw();
}
// Row 2 from the row-1 table: swapping s+ and s- at every point conjugates each influence factor
// (Sec. II, Eq. for I), so lo (x) isum of row 2 at (fl, old) is the conjugate of row 1's at the
// conjugated digits (values 1 <-> 2): sum_old conj(W1[conj old][conj fl]) a[old], flb = conj fl.
__device__ __forceinline__ tf2 conj_tab(tf2 t) {
    t.t1.y = -t.t1.y;
    t.t2.y = -t.t2.y;
    t.t3.y = -t.t3.y;
    return t;
}
__device__ __forceinline__ df2 fold_sum_conj(const FoldRow<QUAPI_DF64>& W, uint32_t flb, const df2 (&a)[4]) {
    dfacc acc;
    acc.init_prod(conj_tab(W.at(0, flb)), a[0]);
    acc.add_prod(conj_tab(W.at(2, flb)), a[1]);
    acc.add_prod(conj_tab(W.at(1, flb)), a[2]);
    acc.add_prod(conj_tab(W.at(3, flb)), a[3]);
    return acc.raw();
}
// Full layout, M = 2, DF64 fast path: rows 1 and 2 through the folded row-1 table
template <int M, int FORM, bool DIAG> __host__ __device__ constexpr bool full_fold() {
    return M == 2 && DIAG && FORM == QUAPI_DF64;
}

// Tables of one launch: summed-digit and lo tables staged in shared memory,
// hi tables read through L1/L2 (256 consecutive fibers share one hi entry).
template <int M, int FORM> struct StepTables {
    using Tab = typename FormT<FORM>::Tab;
    static constexpr int M2 = M * M;
    Tab *isum, *isume, *lo, *loe;
    const Tab *hi, *hie;
    const Tab *w, *we;  // lo (x) isum: [x][f_lo][old], read through L1
    FoldRow<FORM> w1, w1e;  // half layout, folded row 1 (step, readout) in shared memory
    const Tab* r1;  // half layout fast path: row 1 of isum (4 entries) then of lo (256), shared
    uint32_t lo_size;
    int lo_shift;
    int64_t hi_size;

    // shared memory of the half layout's folded variant: W1 for the step and W1e for the readout
    static __host__ __device__ size_t fold_smem_bytes(bool write, bool read) {
        return FoldRow<FORM>::kEntryBytes * ((write ? 1 : 0) + (read ? 1 : 0)) * 4 * (size_t)kFoldLo;
    }
    // shared memory of the half layout's unfolded fast path: row 1 of isum and lo for the step (rows 0
    // and 3 are diagonal there, K only, and row 2 is written from row 1 of the conjugate prefix), and the
    // readout's folded row-1 table (loe (x) isume, formed in FP64 at set-up)
    static __host__ __device__ size_t row1_smem_bytes(int64_t lo_size, bool write, bool read) {
        return (write ? sizeof(Tab) * (M2 + (size_t)lo_size) : 0) + (read ? sizeof(Tab) * 4 * (size_t)kFoldLo : 0);
    }
    template <bool WRITE, bool READ>
    __device__ __forceinline__ void stage_row1(const StepArgs& args, unsigned char* smem) {
        hi = reinterpret_cast<const Tab*>(args.hi);
        hie = reinterpret_cast<const Tab*>(args.hi_e);
        lo_size = (uint32_t)args.lo_size;
        lo_shift = args.lo_shift;
        hi_size = args.F / args.lo_size;
        Tab* bw = reinterpret_cast<Tab*>(smem);
        const Tab* gi = reinterpret_cast<const Tab*>(args.isum);
        const Tab* gl = reinterpret_cast<const Tab*>(args.lo);
        if (WRITE)
            for (uint32_t e = threadIdx.x; e < M2 + lo_size; e += kThreads)
                bw[e] = e < (uint32_t)M2 ? gi[M2 + e] : gl[lo_size + (e - M2)];
        r1 = bw;
        if constexpr (FoldRow<FORM>::kEntryBytes > 0)
            if (READ) w1e.stage(smem + (WRITE ? sizeof(Tab) * (M2 + lo_size) : 0), args.w_e);
    }
    template <bool WRITE, bool READ>
    __device__ __forceinline__ void stage_fold(const StepArgs& args, unsigned char* smem) {
        hi = reinterpret_cast<const Tab*>(args.hi);
        hie = reinterpret_cast<const Tab*>(args.hi_e);
        lo_size = (uint32_t)args.lo_size;
        lo_shift = args.lo_shift;
        hi_size = args.F / args.lo_size;
        if constexpr (FoldRow<FORM>::kEntryBytes > 0) {
            if (WRITE) w1.stage(smem, args.w);
            if (READ) w1e.stage(smem + (WRITE ? fold_smem_bytes(true, false) : 0), args.w_e);
        }
    }

    // shared memory of one variant: isum + lo for the step, isume + loe for the readout
    static __host__ __device__ size_t smem_bytes(int64_t lo_size, bool write, bool read) {
        return sizeof(Tab) * ((write ? 1 : 0) + (read ? 1 : 0)) * (M2 * M2 + M2 * (size_t)lo_size);
    }
    template <bool WRITE, bool READ>
    __device__ __forceinline__ void stage(const StepArgs& args, unsigned char* smem) {
        Tab* base = reinterpret_cast<Tab*>(smem);
        const int64_t one = M2 * M2 + M2 * args.lo_size;
        isum = base;
        lo = base + M2 * M2;
        isume = base + (WRITE ? one : 0);
        loe = isume + M2 * M2;
        hi = reinterpret_cast<const Tab*>(args.hi);
        hie = reinterpret_cast<const Tab*>(args.hi_e);
        w = reinterpret_cast<const Tab*>(args.w);
        we = reinterpret_cast<const Tab*>(args.w_e);
        lo_size = (uint32_t)args.lo_size;
        lo_shift = args.lo_shift;
        hi_size = args.F / args.lo_size;
        const Tab* g_isum = reinterpret_cast<const Tab*>(args.isum);
        const Tab* g_lo = reinterpret_cast<const Tab*>(args.lo);
        const Tab* g_isume = reinterpret_cast<const Tab*>(args.isum_e);
        const Tab* g_loe = reinterpret_cast<const Tab*>(args.lo_e);
        for (int e = threadIdx.x; e < M2 * M2; e += kThreads) {
            if (WRITE) isum[e] = g_isum[e];
            if (READ) isume[e] = g_isume[e];
        }
        for (int e = threadIdx.x; e < M2 * (int)lo_size; e += kThreads) {
            if (WRITE) lo[e] = g_lo[e];
            if (READ) loe[e] = g_loe[e];
        }
    }
};

// All outputs (and readout contributions) of the FPT fibers f0.. held in registers.
// hpre / hepre: the hi entries of this thread's fibers staged by the caller
// (row x at hpre[x * HSTRIDE]; all FPT fibers share one f_hi), or null to load them here.
template <int M, int FORM, bool WRITE, bool READ, bool DIAG, int HSTRIDE = 1>
__device__ __forceinline__ void process_fibers(const StepTables<M, FORM>& T,
                                               typename FormT<FORM>::Elem (&a)[fibers_per_thread<M * M, FORM>()][M * M],
                                               const bool (&valid)[fibers_per_thread<M * M, FORM>()], int64_t f0,
                                               int64_t F,
                                               typename FormT<FORM>::Elem* __restrict__ out,
                                               RhoAcc<FORM> (&racc)[M * M],
                                               const typename FormT<FORM>::Tab* hpre = nullptr,
                                               const typename FormT<FORM>::Tab* hepre = nullptr) {
    constexpr int M2 = M * M;
    using Elem = typename FormT<FORM>::Elem;
    constexpr int FPT = fibers_per_thread<M * M, FORM>();
    uint32_t fhi[FPT], flo[FPT];
#pragma unroll
    for (int u = 0; u < FPT; ++u) Split<M>::split((uint32_t)(f0 + u), T.lo_size, T.lo_shift, fhi[u], flo[u]);

    // diagonal rows: shared plain sum, only K (in hi) applies
    decltype(plain_sum<M2>(a[0])) Sd[FPT];
    if (DIAG) {
#pragma unroll
        for (int u = 0; u < FPT; ++u) Sd[u] = plain_sum<M2>(a[u]);
    }
    // the FPT fibers of a thread share their hi entry when lo_size >= FPT and f0 is a multiple of FPT
    const bool shared_hi = (FPT == 1) || (T.lo_size >= (uint32_t)FPT && fhi[0] == fhi[FPT - 1]);
#pragma unroll
    for (int x = 0; x < M2; ++x) {
        Elem vout[FPT];
        Elem vread[FPT];
        const bool diag_row = DIAG && is_diag<M>(x);
        typename FormT<FORM>::Tab h0, he0;
        if (WRITE) h0 = hpre ? hpre[x * HSTRIDE] : T.hi[(int64_t)x * T.hi_size + fhi[0]];
        if (READ && !(WRITE && diag_row)) he0 = hepre ? hepre[x * HSTRIDE] : T.hie[(int64_t)x * T.hi_size + fhi[0]];
#pragma unroll
        for (int u = 0; u < FPT; ++u) {
            if (!valid[u]) {
                vout[u] = Elem{};
                vread[u] = Elem{};
                continue;
            }
            const bool same = (u == 0) || shared_hi;
            if (diag_row) {
                const int64_t hidx = (int64_t)x * T.hi_size + fhi[u];
                if (WRITE) {
                    vout[u] = apply_hi(same ? h0 : T.hi[hidx], Sd[u]);
                    vread[u] = vout[u];
                } else {
                    vread[u] = apply_hi(same ? he0 : T.hie[hidx], Sd[u]);
                }
            } else {
                if constexpr (FormT<FORM>::kFoldLo) {
                    // w = lo (x) isum folds the lo factor into the sum over the oldest index
                    if (WRITE) {
                        auto S = row_sum<M2>(T.w + ((int64_t)x * T.lo_size + flo[u]) * M2, a[u]);
                        vout[u] = apply_hi(same ? h0 : T.hi[(int64_t)x * T.hi_size + fhi[u]], S);
                    }
                    if (READ) {
                        auto Se = row_sum<M2>(T.we + ((int64_t)x * T.lo_size + flo[u]) * M2, a[u]);
                        vread[u] = apply_hi(same ? he0 : T.hie[(int64_t)x * T.hi_size + fhi[u]], Se);
                    }
                } else if constexpr (full_fold<M, FORM, DIAG>()) {
                    // x = 1 or 2 (the off-diagonal rows): one table product after the folded sum
                    if constexpr (M == 2 && FORM == QUAPI_DF64) {
                        const uint32_t fl = flo[u] & (kFoldLo - 1u);
                        if (WRITE) {
                            const df2 S = (x == 1) ? fold_sum(T.w1, fl, a[u]) : fold_sum_conj(T.w1, conj_digits(fl), a[u]);
                            vout[u] = apply_hi(same ? h0 : T.hi[(int64_t)x * T.hi_size + fhi[u]], S);
                        }
                        if (READ) {
                            const df2 Se =
                                (x == 1) ? fold_sum(T.w1e, fl, a[u]) : fold_sum_conj(T.w1e, conj_digits(fl), a[u]);
                            vread[u] = apply_hi(same ? he0 : T.hie[(int64_t)x * T.hi_size + fhi[u]], Se);
                        }
                    }
                } else {
                    if (WRITE) {
                        auto S = row_sum<M2, DIAG>(T.isum + x * M2, a[u]);
                        vout[u] = apply_p(same ? h0 : T.hi[(int64_t)x * T.hi_size + fhi[u]],
                                          T.lo[x * T.lo_size + flo[u]], S);
                    }
                    if (READ) {
                        auto Se = row_sum<M2, DIAG>(T.isume + x * M2, a[u]);
                        vread[u] = apply_p(same ? he0 : T.hie[(int64_t)x * T.hi_size + fhi[u]],
                                           T.loe[x * T.lo_size + flo[u]], Se);
                    }
                }
            }
            if (READ) racc[x].add(vread[u]);
        }
        if (WRITE) store_row<M, FORM>(out, (int64_t)x * F + f0, vout, valid);
    }
}

// Per-CTA readout partial sums: warp trees, then warp sums in warp order.
template <int M2, int FORM>
__device__ __forceinline__ void write_partials(const RhoAcc<FORM> (&racc)[M2], double2* partial) {
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
        partial[(int64_t)blockIdx.x * M2 + threadIdx.x] = v;
    }
}

// Fused step, plain vectorised global loads (any M, any tensor size).
template <int M, int FORM, bool WRITE, bool READ, bool DIAG>
__global__ void __launch_bounds__(kThreads) step_kernel(StepArgs args) {
    constexpr int M2 = M * M;
    using Elem = typename FormT<FORM>::Elem;
    constexpr int FPT = fibers_per_thread<M2, FORM>();
    constexpr int TILE = kThreads * FPT;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepTables<M, FORM> T;
    if constexpr (full_fold<M, FORM, DIAG>())
        T.template stage_fold<WRITE, READ>(args, smem_raw);
    else
        T.template stage<WRITE, READ>(args, smem_raw);
    __syncthreads();

    RhoAcc<FORM> racc[M2];
#pragma unroll
    for (int x = 0; x < M2; ++x) racc[x].init();

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
        process_fibers<M, FORM, WRITE, READ, DIAG>(T, a, valid, f0, F, out, racc);
    }
    if (READ) write_partials<M2, FORM>(racc, args.partial);
}

// ---- TMA-staged variant (M = 2) -------------------------------------------------
//
// The input tensor is viewed as rows of 128 bytes (4 FP32 fibers or 2 FP64
// fibers per row).  Each tile is one 2-D TMA box of 128 rows (16 KB) loaded
// with the 128-byte swizzle: the 16-byte chunk c of row r lands at chunk
// position c ^ (r mod 8), so that the 8 threads of a quarter warp, each reading
// one 16-byte chunk of its own 64-byte slice, hit 8 different bank groups.
// A ring of STAGES tiles per CTA (one mbarrier each) keeps STAGES x 16 KB of
// loads in flight while the CTA computes and stores; one thread issues the
// copies.  Every wait is bounded (globaltimer, StepArgs::wait_ns); on expiry the CTA records the
// error flag, drains its own copies (bounded) and exits.
constexpr int kTmaRows = 128;
constexpr int kTmaTileBytes = kTmaRows * 128;
constexpr int kBarBytes = 64;                     // mbarrier slot ahead of the tables

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_complete_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_rows(uint32_t dst, const CUtensorMap* map, int32_t row, uint32_t bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

template <int M, int FORM, bool WRITE, bool READ, bool DIAG, int STAGES>
__global__ void __launch_bounds__(kThreads) step_kernel_tma(const __grid_constant__ CUtensorMap in_map,
                                                            StepArgs args) {
    static_assert(M == 2, "the TMA path covers M = 2 (fibers pack whole 128-byte rows)");
    constexpr int M2 = M * M;
    using Elem = typename FormT<FORM>::Elem;
    constexpr int FPT = FormT<FORM>::FPT;
    constexpr int TILE = kThreads * FPT;  // fibers per 16 KB tile
    static_assert(TILE * M2 * (int)sizeof(Elem) == kTmaTileBytes, "tile = one TMA box");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    static_assert(STAGES * 8 <= kBarBytes, "mbarriers fit their slot");
    using Tab = typename FormT<FORM>::Tab;
    // hi entries of one tile: TILE / lo_size (= HPT) consecutive f_hi per row, copied with the tile.
    // They are read after the stage is released, so their ring has one slot more than the tile
    // ring: the refill issued in iteration k overwrites the slot of tile k - 1, never that of tile k.
    constexpr int HPT = TILE / 256;
    constexpr int HSLOTS = STAGES + 1;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + STAGES * kTmaTileBytes);
    Tab* hring = reinterpret_cast<Tab*>(ring + STAGES * kTmaTileBytes + kBarBytes);  // [HSLOTS][2][M2][HPT]
    unsigned char* tables = reinterpret_cast<unsigned char*>(hring + HSLOTS * 2 * M2 * HPT);

    StepTables<M, FORM> T;
    if constexpr (full_fold<M, FORM, DIAG>())
        T.template stage_fold<WRITE, READ>(args, tables);
    else
        T.template stage<WRITE, READ>(args, tables);

    const int64_t F = args.F;
    const int64_t ntiles = F / TILE;
    const int64_t my_tiles = (blockIdx.x < ntiles) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    uint64_t policy = 0;
    const Tab* ghi = reinterpret_cast<const Tab*>(args.hi);
    const Tab* ghie = reinterpret_cast<const Tab*>(args.hi_e);
    const int64_t hi_size = F >> T.lo_shift;
    // one tile: the 16 KB TMA box plus, per row, its HPT hi entries (and the readout's)
    auto issue_tile = [&](int st, int hs, int64_t tile) {
        constexpr uint32_t hb = HPT * sizeof(Tab);
        const uint32_t bytes = kTmaTileBytes + (WRITE ? M2 * hb : 0) + (READ ? M2 * hb : 0);
        const uint32_t bar = smem_u32(&bars[st]);
        // (fault injection only: CTA 0's first tile expects more bytes than arrive, so its wait expires)
        mbar_expect_tx(bar, bytes + ((blockIdx.x == 0 && tile == 0) ? args.fault_tx : 0u));
        tma_load_rows(smem_u32(ring + st * kTmaTileBytes), &in_map, (int32_t)(tile * kTmaRows), bar, policy);
        const int64_t fh0 = tile * HPT;
#pragma unroll
        for (int x = 0; x < M2; ++x) {
            if (WRITE) bulk_load(smem_u32(hring + ((hs * 2 + 0) * M2 + x) * HPT), ghi + x * hi_size + fh0, hb, bar);
            if (READ) bulk_load(smem_u32(hring + ((hs * 2 + 1) * M2 + x) * HPT), ghie + x * hi_size + fh0, hb, bar);
        }
    };
    if (threadIdx.x == 0) {
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
        for (int st = 0; st < STAGES; ++st) mbar_init(smem_u32(&bars[st]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES && st < my_tiles; ++st) {
            const int64_t tile = blockIdx.x + (int64_t)st * gridDim.x;
            issue_tile(st, st % HSLOTS, tile);
        }
    }

    RhoAcc<FORM> racc[M2];
#pragma unroll
    for (int x = 0; x < M2; ++x) racc[x].init();
    Elem* __restrict__ out = reinterpret_cast<Elem*>(args.A_out);

    const int r = threadIdx.x >> 1;            // row of this thread's 64-byte slice
    const int c0 = (threadIdx.x & 1) << 2;     // first of its four 16-byte chunks
    for (int64_t k = 0; k < my_tiles; ++k) {
        const int st = (int)(k % STAGES);
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        const int64_t f0 = (blockIdx.x + k * gridDim.x) * TILE + (int64_t)threadIdx.x * FPT;
        const bool ok = mbar_wait_bounded(smem_u32(&bars[st]), parity, args.wait_ns);
        // this thread's FPT fibers share one f_hi (lo_size = 256 on this path): entry (threadIdx.x * FPT) / 256
        const int hsel = (int)(((int64_t)threadIdx.x * FPT) >> 8);
        const int hs = (int)(k % HSLOTS);
        const Tab* hv = hring + (hs * 2 + 0) * M2 * HPT + hsel;
        const Tab* hve = hring + (hs * 2 + 1) * M2 * HPT + hsel;
        Elem a[FPT][M2];
        if (ok) {
            const unsigned char* row = ring + st * kTmaTileBytes + r * 128;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int pos = (c0 + q) ^ (r & 7);
                if constexpr (FORM == QUAPI_FP32) {
                    const float4 v = *reinterpret_cast<const float4*>(row + pos * 16);
                    const int e0 = 2 * q, e1 = 2 * q + 1;  // entries of the 2-fiber slice
                    a[e0 / M2][e0 % M2] = make_float2(v.x, v.y);
                    a[e1 / M2][e1 % M2] = make_float2(v.z, v.w);
                } else {
                    a[0][q] = *reinterpret_cast<const Elem*>(row + pos * 16);  // one complex entry per chunk
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            // a copy never completed: record it, wait (bounded) for this CTA's
            // copies still in flight, and leave
            if (threadIdx.x == 0) {
                atomicExch(args.err_flag, 1);
                // an injected fault: account for the bytes that never come, so that the drain below
                // waits for the tile's real copies exactly
                if (args.fault_tx && blockIdx.x == 0 && k == 0) mbar_complete_tx(smem_u32(&bars[0]), args.fault_tx);
                for (int64_t j = k; j < my_tiles && j < k + STAGES; ++j)
                    mbar_wait_bounded(smem_u32(&bars[j % STAGES]), (uint32_t)((j / STAGES) & 1), args.wait_ns / 4);
            }
            return;
        }
        // stage st is free again: refill it with tile k + STAGES
        if (threadIdx.x == 0 && k + STAGES < my_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads of the stage before the copy
            const int64_t tile = blockIdx.x + (k + STAGES) * gridDim.x;
            issue_tile(st, (int)((k + STAGES) % HSLOTS), tile);
        }
        bool valid[FPT];
#pragma unroll
        for (int u = 0; u < FPT; ++u) valid[u] = true;
        process_fibers<M, FORM, WRITE, READ, DIAG, HPT>(T, a, valid, f0, F, out, racc, WRITE ? hv : nullptr,
                                                        READ ? hve : nullptr);
    }
    if (READ) write_partials<M2, FORM>(racc, args.partial);
}

// ---- Hermitian half layout (M = 2) ------------------------------------------------
//
// For a Hermitian rho(0), A(conj path) = conj(A(path)) (swapping s+ and s- of
// every point conjugates K and every influence factor).  A prefix is canonical
// when its most significant digit outside {0, 3} is a 1; canonical n-digit
// prefixes are ordered [top 1: 4^(n-1) plain][top 0: canonical n-1][top 3:
// canonical n-1], C(n) = (4^n + 2^n)/2 of them.  An n-digit tensor stores the
// 4-entry last-digit fiber of every canonical (n-1)-digit prefix, prefix c at
// entry 4c (a prefix of only 0s and 3s keeps its redundant digit-2 entry, the
// conjugate of its digit-1 entry).  One thread per canonical input prefix f
// computes, from the one loaded fiber, the rows this layout keeps: (1, f),
// (1, conj f), (0, f), (3, f) (and the conjugate entries (0/3, conj f) when
// those are stored); the readout adds row 1 over f and conj f and twice the
// real part of the diagonal rows (their conjugate partners are conjugates).

// the 4 entries of fiber c (aligned: FP32 as two 16-byte loads)
template <int FORM>
__device__ __forceinline__ void load_fiber4(const typename FormT<FORM>::Elem* __restrict__ A, uint32_t c,
                                            typename FormT<FORM>::Elem (&a)[4]) {
    if constexpr (FORM == QUAPI_FP32) {
        const float4* p = reinterpret_cast<const float4*>(A + 4ull * c);
        const float4 v0 = __ldcs(p), v1 = __ldcs(p + 1);
        a[0] = make_float2(v0.x, v0.y);
        a[1] = make_float2(v0.z, v0.w);
        a[2] = make_float2(v1.x, v1.y);
        a[3] = make_float2(v1.z, v1.w);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = ld_stream(A + 4ull * c + q);
    }
}

// outputs of rows 0, 1, 3 for one fiber a (row 2 is never needed); ONLY1: row 1 alone
template <int FORM, bool DIAG, bool END, bool ONLY1 = false>
__device__ __forceinline__ void herm_rows(const StepTables<2, FORM>& T, const typename FormT<FORM>::Elem (&a)[4],
                                          uint32_t f, typename FormT<FORM>::Elem (&o)[4]) {
    const uint32_t fh = f >> T.lo_shift, fl = f & (T.lo_size - 1u);
    const auto* hi = END ? T.hie : T.hi;
    if constexpr (FormT<FORM>::kFoldLo) {
        const auto* w = END ? T.we : T.w;  // lo (x) isum
        if (ONLY1) {
        } else if (DIAG) {
            const auto S = plain_sum<4>(a);
            o[0] = apply_hi(hi[fh], S);
            o[3] = apply_hi(hi[3 * T.hi_size + fh], S);
        } else {
            o[0] = apply_hi(hi[fh], row_sum<4>(w + (int64_t)fl * 4, a));
            o[3] = apply_hi(hi[3 * T.hi_size + fh], row_sum<4>(w + ((int64_t)3 * T.lo_size + fl) * 4, a));
        }
        o[1] = apply_hi(hi[T.hi_size + fh], row_sum<4>(w + ((int64_t)T.lo_size + fl) * 4, a));
    } else if constexpr (DIAG && herm_fold<FORM>()) {
        // folded row 1 (lo (x) isum staged in shared memory): one table product after the sum;
        // lo_size = 256 here, and hi has hi_size = F / 256 < 2^32 entries per row
        const uint32_t fh8 = f >> 8, hs = (uint32_t)T.hi_size;
        if (!ONLY1) {
            const auto S = plain_sum<4>(a);
            o[0] = apply_hi(hi[fh8], S);
            o[3] = apply_hi(hi[3u * hs + fh8], S);
        }
        o[1] = apply_hi(hi[hs + fh8], fold_sum(END ? T.w1e : T.w1, f & (kFoldLo - 1u), a));
    } else {
        const auto* isum = END ? T.isume : T.isum;
        const auto* lo = END ? T.loe : T.lo;
        if constexpr (herm_row1<FORM, DIAG>()) {  // row 1 of isum and lo staged on their own (stage_row1)
            if (!ONLY1) {
                const auto S = plain_sum<4>(a);
                o[0] = apply_hi(hi[fh], S);
                o[3] = apply_hi(hi[3 * T.hi_size + fh], S);
            }
            if constexpr (END) {  // the readout's folded row-1 table
                o[1] = apply_hi(hi[T.hi_size + (f >> 8)], fold_sum(T.w1e, f & 255u, a));
            } else {  // lo_size = 256 on the fast path
                o[1] = apply_p(hi[T.hi_size + (f >> 8)], T.r1[4 + (f & 255u)], row_sum<4, true>(T.r1, a));
            }
            return;
        }
        if (ONLY1) {
        } else {
            o[0] = apply_p(hi[fh], lo[fl], row_sum<4, DIAG>(isum, a));
            o[3] = apply_p(hi[3 * T.hi_size + fh], lo[3 * T.lo_size + fl], row_sum<4, DIAG>(isum + 12, a));
        }
        o[1] = apply_p(hi[T.hi_size + fh], lo[T.lo_size + fl], row_sum<4, DIAG>(isum + 4, a));
    }
}

// Readout of the FP32 fast path, deferred per hi block.  In a fast chunk every prefix f is its own
// conjugate's canonical partner (no self-conjugate prefixes), and a lane's fibers mostly share their hi
// block fh = f >> 8.  Summed over the fibers of one block, the readout is
//   rho[1] += hie[1][fh] sum W1e[.][fl] a  +  hie[1][conj fh] sum W1e[.][conj fl] b,
//   rho[0 / 3] += 2 Re(hie[0 / 3][fh] sum_f sum_old a),
// so the lane accumulates the three inner sums and multiplies by hie only when fh changes.  The inner
// sums are FP32 products (the hi float of W1e) in FMA chains of at most a block's fibers, of the order
// of the stored data's own rounding (an accumulator for the table's lo floats changed the error against
// the oracle by less than 1e-15 at memory length 14, and cost 6 % more time); each block is added to
// the compensated rho accumulators through one rounded product with the double-float hie.
template <int FORM> struct BlockRead {
    __device__ __forceinline__ void init() {}
};
template <> struct BlockRead<QUAPI_FP32> {
    float2 t1h, tbh, t0;
    uint32_t fh;  // hi block of the sums, ~0u: none
    __device__ __forceinline__ void init() { fh = ~0u; }
    __device__ __forceinline__ void clear() {
        t1h = tbh = t0 = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ static void mac(const ff2& W, float2 v, float2& h) {
        h.x = fmaf(W.hr, v.x, fmaf(-W.hi, v.y, h.x));
        h.y = fmaf(W.hr, v.y, fmaf(W.hi, v.x, h.y));
    }
    __device__ __forceinline__ void flush(const StepTables<2, QUAPI_FP32>& T, RhoAcc<QUAPI_FP32> (&racc)[4]) {
        if (fh == ~0u) return;
        const uint32_t hs = (uint32_t)T.hi_size, fhb = conj_digits(fh);
        racc[1].add(ffmul(T.hie[hs + fh], t1h));
        racc[1].add(ffmul(T.hie[hs + fhb], tbh));
        racc[0].add_re(ffmul(T.hie[fh], t0), 2.f);
        racc[3].add_re(ffmul(T.hie[3u * hs + fh], t0), 2.f);
    }
    __device__ __forceinline__ void add(const StepTables<2, QUAPI_FP32>& T, const float2 (&a)[4],
                                        const float2 (&b)[4], uint32_t f, RhoAcc<QUAPI_FP32> (&racc)[4]) {
        if ((f >> 8) != fh) {
            flush(T, racc);
            fh = f >> 8;
            clear();
        }
        const uint32_t fl = f & 255u, flb = conj_digits(fl);
#pragma unroll
        for (int q = 0; q < 4; ++q) mac(T.w1e.at(q, fl), a[q], t1h);
#pragma unroll
        for (int q = 0; q < 4; ++q) mac(T.w1e.at(q, flb), b[q], tbh);
        t0.x += (a[0].x + a[1].x) + (a[2].x + a[3].x);
        t0.y += (a[0].y + a[1].y) + (a[2].y + a[3].y);
    }
};
template <int FORM, bool DIAG> __host__ __device__ constexpr bool herm_block_read() {
    return herm_row1<FORM, DIAG>() && FORM == QUAPI_FP32;
}

// Everything one canonical input prefix f contributes: its decoded plain digits f, whether f is its
// own conjugate (sc), the canonical position h of fh = f >> 2 and whether fh is its own conjugate (shc).
// The store position h (and shc) is found after the rows are computed, which keeps it out of the
// arithmetic's live range: given (hfast, shc = false) when known, else decoded from f.
template <int FORM, bool WRITE, bool READ, bool DIAG>
__device__ __forceinline__ void herm_fiber(const StepTables<2, FORM>& T, const typename FormT<FORM>::Elem (&a)[4],
                                           uint32_t f, bool sc, bool known, uint32_t hfast, int np, uint32_t top,
                                           uint32_t cnh, typename FormT<FORM>::Elem* __restrict__ out,
                                           RhoAcc<FORM> (&racc)[4], BlockRead<FORM>& blk) {
    using Elem = typename FormT<FORM>::Elem;
    constexpr int remap[4] = {0, 2, 1, 3};
    Elem b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = conjv(a[remap[q]]);  // fiber of the conjugate prefix
    const uint32_t fb = conj_digits(f);
    if (WRITE) {
        Elem o[4];
        herm_rows<FORM, DIAG, false>(T, a, f, o);
        if (np == 0) {  // one-digit output: every point stored
            st_stream(out + 0, o[0]);
            st_stream(out + 1, o[1]);
            st_stream(out + 2, conjv(o[1]));
            st_stream(out + 3, o[3]);
        } else {
            const uint32_t fl = f & 3u;
            const uint32_t h = known ? hfast : half_position(f >> 2, np - 1);
            const bool shc = known ? false : self_conjugate(f >> 2, np - 1);
            const uint32_t b0 = 4u * (top + h), b3 = 4u * (top + cnh + h);
            st_stream(out + f, o[1]);
            st_stream(out + b0 + fl, o[0]);
            st_stream(out + b3 + fl, o[3]);
            if (!sc) {
                Elem ob[4];
                herm_rows<FORM, DIAG, false, true>(T, b, fb, ob);
                st_stream(out + fb, ob[1]);
                if (shc) {  // (0/3, fh, 2) are stored too: conjugates of (0/3, f)
                    st_stream(out + b0 + 2, conjv(o[0]));
                    st_stream(out + b3 + 2, conjv(o[3]));
                }
            }
        }
    }
    if (READ) {
        if constexpr (herm_block_read<FORM, DIAG>()) {
            if (known) {  // fast chunk: deferred per hi block
                blk.add(T, a, b, f, racc);
                return;
            }
        }
        Elem r[4];
        herm_rows<FORM, DIAG, true>(T, a, f, r);
        racc[1].add(r[1]);
        if (!sc) {
            Elem rb[4];
            herm_rows<FORM, DIAG, true, true>(T, b, fb, rb);
            racc[1].add(rb[1]);
            racc[0].add_re(r[0], 2);  // rows 0 and 3: the conjugate partner adds the conjugate
            racc[3].add_re(r[3], 2);
        } else {
            racc[0].add_re(r[0], 1);
            racc[3].add_re(r[3], 1);
        }
    }
}

// Work is handed out in warp chunks of consecutive canonical positions (chunk / 32 per lane): 256
// positions when the tensor is large enough to give every resident warp several chunks, fewer (down
// to 32) for smaller tensors so that every warp still gets work.
// Nearly every chunk lies inside one digit-1 block of level >= 2 (all but the last few levels):
// it is decoded once and its prefixes are then consecutive plain indices, f = f0 + i with fiber
// position h = h0 + i / 4.  Other chunks decode each position on its own.
constexpr uint32_t kChunk = 256;

// Minimum resident CTAs per SM given to the compiler (a register cap).  Measured at memory length 14:
// the FP32 step runs best at 8 CTAs (32 registers; 0.370 ms against 0.380 ms at 6 CTAs and
// 0.425 ms uncapped), the FP32 step with the per-block readout at 4 (64 registers, no spills;
// 0.561 ms, 0.562 at 3); the readout alone, and the DF64 and FP64 forms, at 3-4.
template <int FORM, bool WRITE, bool READ> constexpr int herm_min_ctas() {
    if (FORM == QUAPI_FP32) return (WRITE && !READ) ? 8 : 4;
    if (WRITE && READ) return 3;
    return (FORM == QUAPI_DF64 && READ) ? 3 : 4;
}

template <int FORM, bool WRITE, bool READ, bool DIAG>
__global__ void __launch_bounds__(kThreads, herm_min_ctas<FORM, WRITE, READ>()) herm_step_kernel(StepArgs args) {
    using Elem = typename FormT<FORM>::Elem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_allow_next();
    StepTables<2, FORM> T;
    if constexpr (DIAG && herm_fold<FORM>())
        T.template stage_fold<WRITE, READ>(args, smem_raw);
    else if constexpr (herm_row1<FORM, DIAG>())
        T.template stage_row1<WRITE, READ>(args, smem_raw);
    else
        T.template stage<WRITE, READ>(args, smem_raw);
    __syncthreads();
    pdl_wait();  // the tables are set-up data; the tensor and the partials belong to the previous kernel
    RhoAcc<FORM> racc[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) racc[x].init();
    BlockRead<FORM> blk;
    blk.init();
    const Elem* __restrict__ A = reinterpret_cast<const Elem*>(args.A_in);
    Elem* __restrict__ out = reinterpret_cast<Elem*>(args.A_out);
    const int np = args.half_digits;           // digits of the prefix f (n_in - 1); 32-bit indices (np <= 15)
    const uint32_t npre = half_count32(np);
    const uint32_t top = (np >= 1) ? (1u << (2 * (np - 1))) : 0u;   // 4^(np-1)
    const uint32_t cnh = (np >= 1) ? half_count32(np - 1) : 0u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = gridDim.x * (kThreads / 32);
    const uint32_t chunk = min(kChunk, max(32u, ((npre + nwarps - 1) / nwarps + 31u) & ~31u));
#pragma unroll 1
    for (uint32_t cb = (blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5)) * chunk; cb < npre;
         cb += nwarps * chunk) {
        uint32_t fb0, hb0;
        bool sc0, shc0;
        half_decode_pair(cb, np, fb0, sc0, hb0, shc0);
        // r1 = 4^(level - 1) of the chunk's digit-1 block (the lowest bit of f's top digit outside {0, 3});
        // the chunk stays inside it when fb0's offset in the block + chunk <= r1 (fb0 a multiple of 4)
        const uint32_t t = (fb0 ^ (fb0 >> 1)) & 0x55555555u;
        const uint32_t r1 = t ? (1u << (31 - __clz(t))) : 0u;
        const bool fast = !sc0 && !shc0 && (fb0 & 3u) == 0u && (fb0 & (r1 - 1u)) + chunk <= r1;
#pragma unroll 1
        for (uint32_t i = lane; i < chunk; i += 32) {
            const uint32_t c = cb + i;
            if (c >= npre) break;
            Elem a[4];
            load_fiber4<FORM>(A, c, a);
            uint32_t f;
            bool sc;
            if (fast) {
                f = fb0 + i;
                sc = false;
            } else {
                half_decode(c, np, f, sc);
            }
            herm_fiber<FORM, WRITE, READ, DIAG>(T, a, f, sc, fast, hb0 + (i >> 2), np, top, cnh, out, racc, blk);
        }
    }
    if constexpr (READ && herm_block_read<FORM, DIAG>()) blk.flush(T, racc);
    if (READ) {
        // row 2 of rho is the conjugate of row 1
        __shared__ double2 red[kThreads / 32][4];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            if (x == 2) continue;
            double2 v = racc[x].value();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, off);
                v.y += __shfl_down_sync(0xffffffffu, v.y, off);
            }
            if (lane == 0) red[warp][x] = v;
        }
        __syncthreads();
        if (threadIdx.x < 4 && threadIdx.x != 2) {
            double2 v = make_double2(0.0, 0.0);
            for (int w = 0; w < kThreads / 32; ++w) v = cadd(v, red[w][threadIdx.x]);
            args.partial[(int64_t)blockIdx.x * 4 + threadIdx.x] = v;
            if (threadIdx.x == 1) args.partial[(int64_t)blockIdx.x * 4 + 2] = make_double2(v.x, -v.y);
        }
    }
}

// ---- Hermitian half layout, M = 3 ---------------------------------------------------------------
//
// Points x = 3a + b; conjugation (a, b) -> (b, a) swaps 1 <-> 3, 2 <-> 6, 5 <-> 7 and keeps 0, 4, 8
// (layout and index helpers in half_layout.cuh).  One thread per canonical input prefix f (np digits)
// computes all nine rows of its fiber and stores what the layout keeps:
//   rows 1, 2, 5 (canonical tops, blocks t = 0, 1, 2 of 9^np plain entries): out[t 9^np + f];
//   rows 3, 6, 7: rows 1, 2, 5 of the conjugate prefix, conjugated, at out[t 9^np + conj f]
//     (f not its own conjugate);
//   rows 0, 4, 8 (self-conjugate tops, t' = 0, 1, 2): the fiber of the prefix (x, f / 9) at
//     9 (9^np / 3 + t' C3(np - 1) + h) + f % 9, h = canonical position of f / 9; when f / 9 is its
//     own conjugate that fiber keeps every last digit, and entry conj(f % 9) is the conjugate value.
// The readout adds r_x + conj(r_conj x) for x = 1, 2, 5 (r_x alone when f is its own conjugate) and
// 2 Re r_x (Re r_x) for x = 0, 4, 8; rows 3, 6, 7 of rho are the conjugates of rows 1, 2, 5.

template <int FORM>
__device__ __forceinline__ void load_fiber9(const typename FormT<FORM>::Elem* __restrict__ A, uint32_t c,
                                            typename FormT<FORM>::Elem (&a)[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) a[q] = ld_stream(A + 9ull * c + q);
}

// The sum over the oldest index of row x, multiplied by lo (FP64: the folded lo (x) isum sum): the row
// is then hi[x][fh] times it (step tables, or the readout's with END).
template <int FORM, bool END, bool DIAG>
__device__ __forceinline__ auto lo_sum9(const StepTables<3, FORM>& T, const typename FormT<FORM>::Elem (&a)[9], int x,
                                        uint32_t fl) {
    if constexpr (FormT<FORM>::kFoldLo) {
        const auto* w = END ? T.we : T.w;  // lo (x) isum
        return row_sum<9>(w + ((int64_t)x * T.lo_size + fl) * 9, a);
    } else if constexpr (FORM == QUAPI_FP32) {
        const kahan32 S = row_sum<9, DIAG>((END ? T.isume : T.isum) + x * 9, a);
        return ffmul2((END ? T.loe : T.lo)[x * T.lo_size + fl], S.s, S.c);
    } else {
        return tfmul((END ? T.loe : T.lo)[x * T.lo_size + fl], row_sum<9>((END ? T.isume : T.isum) + x * 9, a));
    }
}

// Rows are formed one at a time and stored (or added to the readout) at once, so that only the fiber
// and one row are live.  The influence factors of the summed and the lo digits depend on the new
// point x only through d(x) = s_a - s_b (Sec. II, Eq. for I; K sits in hi on the fast path), so for
// equally spaced coordinate eigenvalues (EQS: s_1 - s_0 = s_2 - s_1) rows 1 and 5 (d = s_0 - s_1) and
// rows 3 and 7 (d = s_1 - s_0) have equal isum and lo rows and share that part of the work.
template <int FORM, bool WRITE, bool READ, bool DIAG, bool EQS>
__device__ __forceinline__ void herm3_fiber(const StepTables<3, FORM>& T, const typename FormT<FORM>::Elem (&a)[9],
                                            uint32_t f, uint32_t fb, bool sc, uint32_t h, bool shc, int np, uint32_t P1,
                                            uint32_t sbase, uint32_t cnh, typename FormT<FORM>::Elem* __restrict__ out,
                                            RhoAcc<FORM> (&racc)[9]) {
    using Elem = typename FormT<FORM>::Elem;
    constexpr bool SHARE = EQS && DIAG;
    constexpr int order[9] = {1, 5, 3, 7, 2, 6, 0, 4, 8};  // the sharing pairs next to each other
    uint32_t fh, fl;
    Split<3>::split(f, T.lo_size, T.lo_shift, fh, fl);
    decltype(plain_sum<9>(a)) Sd;
    if (DIAG) Sd = plain_sum<9>(a);
    if (WRITE) {
        const uint32_t f0 = f % 9u;
        const uint32_t e0 = 9u * (sbase + h) + f0;  // rows 0, 4, 8: their fibers are C3(np - 1) prefixes apart
        const uint32_t e1 = e0 - f0 + conj3(f0);
        decltype(lo_sum9<FORM, false, DIAG>(T, a, 0, fl)) ls;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int x = order[k];
            const auto hx = T.hi[(int64_t)x * T.hi_size + fh];
            Elem v;
            if (DIAG && is_diag<3>(x)) {
                v = apply_hi(hx, Sd);
            } else {
                if (!(SHARE && (x == 5 || x == 7))) ls = lo_sum9<FORM, false, DIAG>(T, a, x, fl);
                v = tmul(hx, ls);
            }
            if (np == 0) {  // one-digit output: every point stored
                st_stream(out + x, v);
                continue;
            }
            if (x == 1 || x == 2 || x == 5) {
                st_stream(out + (x == 1 ? 0u : (x == 2 ? P1 : 2u * P1)) + f, v);
            } else if (x == 3 || x == 6 || x == 7) {  // rows 1, 2, 5 of the conjugate prefix
                if (!sc) st_stream(out + (x == 3 ? 0u : (x == 6 ? P1 : 2u * P1)) + fb, conjv(v));
            } else {
                const uint32_t off = (x == 0 ? 0u : (x == 4 ? 9u * cnh : 18u * cnh));
                st_stream(out + e0 + off, v);
                if (!sc && shc) st_stream(out + e1 + off, conjv(v));  // self-conjugate (x, f / 9): every last digit
            }
        }
    }
    if (READ) {
        decltype(lo_sum9<FORM, true, DIAG>(T, a, 0, fl)) ls;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int x = order[k];
            const auto hx = T.hie[(int64_t)x * T.hi_size + fh];
            Elem r;
            if (DIAG && is_diag<3>(x)) {
                r = apply_hi(hx, Sd);
            } else {
                if (!(SHARE && (x == 5 || x == 7))) ls = lo_sum9<FORM, true, DIAG>(T, a, x, fl);
                r = tmul(hx, ls);
            }
            if (x == 1 || x == 2 || x == 5) {
                racc[x].add(r);
            } else if (x == 3 || x == 6 || x == 7) {
                if (!sc) racc[conj3(x)].add(conjv(r));
            } else {
                racc[x].add_re(r, sc ? 1 : 2);
            }
        }
    }
}

// Minimum resident CTAs per SM given to the compiler (nine-entry fibers: many live values)
template <int FORM, bool WRITE, bool READ> constexpr int herm3_min_ctas() {
    return (FORM == QUAPI_FP32 && WRITE && !READ) ? 3 : 2;
}

template <int FORM, bool WRITE, bool READ, bool DIAG, bool EQS>
__global__ void __launch_bounds__(kThreads, herm3_min_ctas<FORM, WRITE, READ>()) herm3_step_kernel(StepArgs args) {
    using Elem = typename FormT<FORM>::Elem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepTables<3, FORM> T;
    T.template stage<WRITE, READ>(args, smem_raw);
    __syncthreads();
    RhoAcc<FORM> racc[9];
#pragma unroll
    for (int x = 0; x < 9; ++x) racc[x].init();
    const Elem* __restrict__ A = reinterpret_cast<const Elem*>(args.A_in);
    Elem* __restrict__ out = reinterpret_cast<Elem*>(args.A_out);
    const int np = args.half_digits;  // digits of the prefix f (n_in - 1); base-9 indices in 32 bits
    const uint32_t npre = half3_count(np);
    const uint32_t P1 = pow9(np);                          // plain block of a canonical top in the output
    const uint32_t sbase = (np >= 1) ? P1 / 3u : 0u;       // 3 x 9^(np-1): first self-conjugate output prefix
    const uint32_t cnh = (np >= 1) ? half3_count(np - 1) : 0u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = gridDim.x * (kThreads / 32);
    const uint32_t chunk = min(kChunk, max(32u, ((npre + nwarps - 1) / nwarps + 31u) & ~31u));
    uint32_t qc = ~0u, cq = 0;  // fast path: the conjugate of f / 81 (digits above the last two), per lane
#pragma unroll 1
    for (uint32_t cb = (blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5)) * chunk; cb < npre;
         cb += nwarps * chunk) {
        // a chunk inside one plain block of a canonical top digit (level >= 2) is decoded once: its
        // prefixes are consecutive plain indices, and so are the positions of their f / 9
        uint32_t fb0, hb0, run;
        bool sc0, shc0;
        half3_decode_run(cb, np, fb0, sc0, hb0, shc0, run);
        const bool fast = run >= min(chunk, npre - cb);
        const uint32_t r0 = fb0 % 9u;
#pragma unroll 1
        for (uint32_t i = lane; i < chunk; i += 32) {
            const uint32_t c = cb + i;
            if (c >= npre) break;
            Elem a[9];
            load_fiber9<FORM>(A, c, a);
            uint32_t f, h, fb;
            bool sc, shc;
            if (fast) {  // np >= 2 here
                f = fb0 + i;
                h = hb0 + (r0 + i) / 9u;
                sc = false;
                shc = false;
                const uint32_t qf = f / 81u, r = f - 81u * qf;
                if (qf != qc) {
                    qc = qf;
                    cq = 81u * conj_digits3(qf, np - 2);
                }
                fb = cq + 9u * conj3(r / 9u) + conj3(r % 9u);
            } else {
                half3_decode_pair(c, np, f, sc, h, shc);
                fb = sc ? f : conj_digits3(f, np);
            }
            herm3_fiber<FORM, WRITE, READ, DIAG, EQS>(T, a, f, fb, sc, h, shc, np, P1, sbase, cnh, out, racc);
        }
    }
    if (READ) {
        // rows 3, 6, 7 of rho are the conjugates of rows 1, 2, 5
        __shared__ double2 red[kThreads / 32][9];
        const int wl = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int x = 0; x < 9; ++x) {
            if (x == 3 || x == 6 || x == 7) continue;
            double2 v = racc[x].value();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, off);
                v.y += __shfl_down_sync(0xffffffffu, v.y, off);
            }
            if (wl == 0) red[warp][x] = v;
        }
        __syncthreads();
        const int x = threadIdx.x;
        if (x < 9 && x != 3 && x != 6 && x != 7) {
            double2 v = make_double2(0.0, 0.0);
            for (int w = 0; w < kThreads / 32; ++w) v = cadd(v, red[w][x]);
            args.partial[(int64_t)blockIdx.x * 9 + x] = v;
            if (x == 1 || x == 2 || x == 5) args.partial[(int64_t)blockIdx.x * 9 + conj3(x)] = make_double2(v.x, -v.y);
        }
    }
}

// growth in the M = 3 half layout: input n_in digits -> n_in + 1 digits, one thread per stored entry
// e = 9 c + d of canonical (or self-conjugate) input prefix c.  With i = (P, d) the plain input index:
// rows 1, 2, 5 at i in their plain blocks (unless P is its own conjugate and d is 3, 6 or 7: that entry
// is the conjugate write of (P, conj d)); rows 3, 6, 7 as rows 1, 2, 5 at conj i with conj A (unless P
// is its own conjugate and d is not 1, 2 or 5: i is self-conjugate, or the write is (P, conj d)'s);
// rows 0, 4, 8 at the fiber of the prefix (x, P), entry d.
template <int FORM>
__global__ void __launch_bounds__(kThreads) herm3_grow_kernel(const void* __restrict__ A_in_, void* __restrict__ A_out_,
                                                              int n_in, const void* __restrict__ lo_,
                                                              const void* __restrict__ hi_, int64_t lo_size_) {
    using Elem = typename FormT<FORM>::Elem;
    using Tab = typename FormT<FORM>::Tab;
    const Elem* A = reinterpret_cast<const Elem*>(A_in_);
    Elem* out = reinterpret_cast<Elem*>(A_out_);
    const Tab* lo = reinterpret_cast<const Tab*>(lo_);
    const Tab* hi = reinterpret_cast<const Tab*>(hi_);
    const uint32_t S = pow9(n_in);              // plain block of a canonical top in the output
    const uint32_t Cp = half3_count(n_in - 1);  // canonical prefixes of the input
    const uint32_t sbase = S / 3u;              // 3 x 9^(n_in - 1)
    const uint32_t lo_size = (uint32_t)lo_size_;
    const int64_t hi_size = S / lo_size;
    const int64_t entries = 9 * (int64_t)Cp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(e / 9), d = (uint32_t)(e % 9);
        uint32_t P;
        bool scP;
        half3_decode(c, n_in - 1, P, scP);
        const uint32_t i = P * 9u + d;
        const Elem v = A[e];
        auto Pm = [&](int x, uint32_t idx, Elem w) {
            return tmul(hi[(int64_t)x * hi_size + idx / lo_size], tmul(lo[(int64_t)x * lo_size + idx % lo_size], w));
        };
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

// growth in the half layout: input n_in digits -> n_in + 1 digits, one thread per stored entry
template <int FORM>
__global__ void __launch_bounds__(kThreads) herm_grow_kernel(const void* __restrict__ A_in_, void* __restrict__ A_out_,
                                                             int n_in, const void* __restrict__ lo_,
                                                             const void* __restrict__ hi_, int64_t lo_size_,
                                                             int lo_shift) {
    using Elem = typename FormT<FORM>::Elem;
    using Tab = typename FormT<FORM>::Tab;
    const Elem* A = reinterpret_cast<const Elem*>(A_in_);
    Elem* out = reinterpret_cast<Elem*>(A_out_);
    const Tab* lo = reinterpret_cast<const Tab*>(lo_);
    const Tab* hi = reinterpret_cast<const Tab*>(hi_);
    const int64_t S = int64_t(1) << (2 * n_in);          // plain row-1 block of the output
    const int64_t Cp = half_count(n_in - 1);             // canonical prefixes of the input
    const int64_t entries = 4 * Cp;
    const uint32_t lo_size = (uint32_t)lo_size_;
    const int64_t hi_size = S / lo_size_;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e >> 2;
        const uint32_t d = (uint32_t)(e & 3);
        uint32_t P;
        bool scP;
        half_decode((uint32_t)c, n_in - 1, P, scP);
        const uint32_t i = (P << 2) | d;
        const Elem v = A[e];
        auto Pm = [&](int x, uint32_t idx, Elem w) {
            return tmul(hi[(int64_t)x * hi_size + (idx >> lo_shift)], tmul(lo[(int64_t)x * lo_size + (idx & (lo_size - 1u))], w));
        };
        if (!(scP && d == 2u)) {  // (P, 2) of a self-conjugate P is written from (P, 1)
            out[i] = Pm(1, i, v);
            if (!(scP && (d == 0u || d == 3u))) {
                const uint32_t ib = conj_digits(i);
                out[ib] = Pm(1, ib, conjv(v));
            }
        }
        out[4 * ((S >> 2) + c) + d] = Pm(0, i, v);
        out[4 * ((S >> 2) + Cp + c) + d] = Pm(3, i, v);
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

// rho_out[x] = the sum of the nparts per-CTA partials of entry x (stored [part][x]), in a fixed order
// that does not depend on timing: thread t of the 32 M2 adds, in turn, the partials j, j + 32, j + 64,
// ... of entry x = t % M2 (j = t / M2; consecutive threads read consecutive partials), then thread x
// adds the 32 sums of its entry in the order j = 0..31.
constexpr int kReduceLanes = 32;
__global__ void __launch_bounds__(kReduceLanes * 9) rho_reduce_kernel(const double2* __restrict__ partial,
                                                                       int nparts, int M2,
                                                                       double2* __restrict__ rho_out) {
    __shared__ double2 sums[kReduceLanes * 9];
    const int t = threadIdx.x, x = t % M2, j = t / M2;
    double2 v = make_double2(0.0, 0.0);
#pragma unroll 4
    for (int b = j; b < nparts; b += kReduceLanes) v = cadd(v, partial[(int64_t)b * M2 + x]);
    sums[t] = v;
    __syncthreads();
    if (t < M2) {
        double2 r = sums[t];
        for (int k = 1; k < kReduceLanes; ++k) r = cadd(r, sums[k * M2 + t]);
        rho_out[t] = r;
    }
}

template <int M, int FORM, bool W, bool R, bool D>
cudaError_t launch_variant(StepArgs& a, cudaStream_t st) {
    constexpr int FPT = fibers_per_thread<M * M, FORM>();
    constexpr bool fold = full_fold<M, FORM, D>();
    if (fold && a.lo_size != kFoldLo) return cudaErrorInvalidValue;  // the fast path resolves 4 lo digits
    size_t smem = fold ? StepTables<M, FORM>::fold_smem_bytes(W, R) : StepTables<M, FORM>::smem_bytes(a.lo_size, W, R);
    auto kern = step_kernel<M, FORM, W, R, D>;
    if (smem > 40 * 1024) {  // the default 48 KB includes the static shared memory
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

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D view of a tensor as rows of 32 four-byte words (128 B), 128-row boxes, 128-byte swizzle.
bool encode_rows_map(CUtensorMap* map, const void* base, int64_t bytes) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || bytes % (128 * kTmaRows) != 0) return false;
    const int64_t rows = bytes / 128;
    if (rows > (int64_t(1) << 32)) return false;
    cuuint64_t dims[2] = {32, (cuuint64_t)rows};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {32, (cuuint32_t)kTmaRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int FORM, bool W, bool R, bool D, int STAGES>
cudaError_t launch_tma_variant(StepArgs& a, const CUtensorMap& map, cudaStream_t st) {
    constexpr int HPT = (kThreads * FormT<FORM>::FPT) / 256;
    size_t smem = 1024 + (size_t)STAGES * kTmaTileBytes + kBarBytes +
                  (size_t)(STAGES + 1) * 2 * 4 * HPT * sizeof(typename FormT<FORM>::Tab) +
                  (full_fold<2, FORM, D>() ? StepTables<2, FORM>::fold_smem_bytes(W, R)
                                           : StepTables<2, FORM>::smem_bytes(a.lo_size, W, R));
    auto kern = step_kernel_tma<2, FORM, W, R, D, STAGES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    constexpr int FPT = FormT<FORM>::FPT;
    const int64_t ntiles = a.F / ((int64_t)kThreads * FPT);
    int64_t g = (int64_t)num_sms() * occ;
    if (g > ntiles) g = ntiles;
    if (g > a.grid) g = a.grid;
    if (g < 1) g = 1;
    a.grid = (int)g;
    kern<<<a.grid, kThreads, smem, st>>>(map, a);
    count_launch();
    return cudaGetLastError();
}

template <int FORM, bool W, bool R, bool D>
cudaError_t launch_tma_stages(StepArgs& a, const CUtensorMap& map, cudaStream_t st) {
    switch (a.stages) {
        case 2: return launch_tma_variant<FORM, W, R, D, 2>(a, map, st);
        case 3: return launch_tma_variant<FORM, W, R, D, 3>(a, map, st);
        case 6: return launch_tma_variant<FORM, W, R, D, 6>(a, map, st);
        default: return launch_tma_variant<FORM, W, R, D, 4>(a, map, st);
    }
}

template <int M, int FORM>
cudaError_t launch_step_mf(StepArgs& a, cudaStream_t st) {
    const bool W = a.A_out != nullptr, R = a.partial != nullptr;
    if constexpr (M == 2) if (a.use_tma && a.diag_fast && a.lo_size == 256) {
        constexpr int FPT = FormT<FORM>::FPT;
        const int64_t elt = (FORM == QUAPI_FP32) ? 8 : 16;
        CUtensorMap map;
        if (a.F % ((int64_t)kThreads * FPT) == 0 && encode_rows_map(&map, a.A_in, a.F * M * M * elt)) {
            if (W && R) return launch_tma_stages<FORM, true, true, true>(a, map, st);
            if (W) return launch_tma_stages<FORM, true, false, true>(a, map, st);
            if (R) return launch_tma_stages<FORM, false, true, true>(a, map, st);
        }
    }
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
    if (M == 2 && form == QUAPI_DF64) return launch_step_mf<2, QUAPI_DF64>(a, st);
    if (M == 3 && form == QUAPI_DF64) return launch_step_mf<3, QUAPI_DF64>(a, st);
    return cudaErrorInvalidValue;
}

namespace {
template <int FORM, bool W, bool R, bool D>
cudaError_t launch_herm_variant(StepArgs& a, cudaStream_t st) {
    constexpr bool fold = D && herm_fold<FORM>();
    if (fold && a.lo_size != kFoldLo) return cudaErrorInvalidValue;  // the fast path resolves 4 lo digits
    size_t smem = fold                      ? StepTables<2, FORM>::fold_smem_bytes(W, R)
                  : herm_row1<FORM, D>() ? StepTables<2, FORM>::row1_smem_bytes(a.lo_size, W, R)
                                          : StepTables<2, FORM>::smem_bytes(a.lo_size, W, R);
    auto kern = herm_step_kernel<FORM, W, R, D>;
    if (smem > 40 * 1024) {  // above the default 48 KB once the kernel's static shared memory is added
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t work = (half_count(a.half_digits) + kThreads - 1) / kThreads;
    int64_t g = (int64_t)num_sms() * (occ < 1 ? 1 : occ);
    if (g > work) g = work;
    if (g > a.grid) g = a.grid;
    if (g < 1) g = 1;
    a.grid = (int)g;
    // programmatic dependent launch where it measured faster: tensors of memory length <= 12 (at most
    // 2^23 canonical prefixes), whose steps are short enough for the launch gap and the table staging
    // to count (spin_boson_L6 0.346 -> 0.262 ms per propagation, quantum dot 10.16 -> 9.86 ms); at
    // memory length 14 it cost 0.5 %
    e = launch_pdl(kern, a.grid, smem, st, a, half_count(a.half_digits) <= (int64_t(1) << 23));
    count_launch();
    return e;
}
template <int FORM>
cudaError_t launch_herm_form(StepArgs& a, cudaStream_t st) {
    const bool W = a.A_out != nullptr, R = a.partial != nullptr;
    if (a.diag_fast) {
        if (W && R) return launch_herm_variant<FORM, true, true, true>(a, st);
        if (W) return launch_herm_variant<FORM, true, false, true>(a, st);
        if (R) return launch_herm_variant<FORM, false, true, true>(a, st);
    } else {
        if (W && R) return launch_herm_variant<FORM, true, true, false>(a, st);
        if (W) return launch_herm_variant<FORM, true, false, false>(a, st);
        if (R) return launch_herm_variant<FORM, false, true, false>(a, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_herm_step(int form, StepArgs& a, cudaStream_t st) {
    if (form == QUAPI_FP64) return launch_herm_form<QUAPI_FP64>(a, st);
    if (form == QUAPI_FP32) return launch_herm_form<QUAPI_FP32>(a, st);
    if (form == QUAPI_DF64) return launch_herm_form<QUAPI_DF64>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_herm_grow(int form, const void* A_in, void* A_out, int n_in, const void* lo, const void* hi,
                             int64_t lo_size, int lo_shift, cudaStream_t st) {
    const int64_t Cn = half_entries(n_in);
    int64_t blocks = (Cn + kThreads - 1) / kThreads;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    if (blocks < 1) blocks = 1;
    if (form == QUAPI_FP64)
        herm_grow_kernel<QUAPI_FP64><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size, lo_shift);
    else if (form == QUAPI_FP32)
        herm_grow_kernel<QUAPI_FP32><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size, lo_shift);
    else if (form == QUAPI_DF64)
        herm_grow_kernel<QUAPI_DF64><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size, lo_shift);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

namespace {
template <int FORM, bool W, bool R, bool D, bool EQS = false>
cudaError_t launch_herm3_variant(StepArgs& a, cudaStream_t st) {
    const size_t smem = StepTables<3, FORM>::smem_bytes(a.lo_size, W, R);
    auto kern = herm3_step_kernel<FORM, W, R, D, EQS>;
    if (smem > 40 * 1024) {  // the default 48 KB includes the static shared memory
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t work = ((int64_t)half3_count(a.half_digits) + kThreads - 1) / kThreads;
    int64_t g = (int64_t)num_sms() * (occ < 1 ? 1 : occ);
    if (g > work) g = work;
    if (g > a.grid) g = a.grid;
    if (g < 1) g = 1;
    a.grid = (int)g;
    kern<<<a.grid, kThreads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}
template <int FORM>
cudaError_t launch_herm3_form(StepArgs& a, cudaStream_t st) {
    const bool W = a.A_out != nullptr, R = a.partial != nullptr;
    if (a.diag_fast && a.eq_spaced) {
        if (W && R) return launch_herm3_variant<FORM, true, true, true, true>(a, st);
        if (W) return launch_herm3_variant<FORM, true, false, true, true>(a, st);
        if (R) return launch_herm3_variant<FORM, false, true, true, true>(a, st);
    } else if (a.diag_fast) {
        if (W && R) return launch_herm3_variant<FORM, true, true, true>(a, st);
        if (W) return launch_herm3_variant<FORM, true, false, true>(a, st);
        if (R) return launch_herm3_variant<FORM, false, true, true>(a, st);
    } else {
        if (W && R) return launch_herm3_variant<FORM, true, true, false>(a, st);
        if (W) return launch_herm3_variant<FORM, true, false, false>(a, st);
        if (R) return launch_herm3_variant<FORM, false, true, false>(a, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_herm3_step(int form, StepArgs& a, cudaStream_t st) {
    if (form == QUAPI_FP64) return launch_herm3_form<QUAPI_FP64>(a, st);
    if (form == QUAPI_FP32) return launch_herm3_form<QUAPI_FP32>(a, st);
    if (form == QUAPI_DF64) return launch_herm3_form<QUAPI_DF64>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_herm3_grow(int form, const void* A_in, void* A_out, int n_in, const void* lo, const void* hi,
                              int64_t lo_size, cudaStream_t st) {
    const int64_t Cn = half3_entries(n_in);
    int64_t blocks = (Cn + kThreads - 1) / kThreads;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    if (blocks < 1) blocks = 1;
    if (form == QUAPI_FP64)
        herm3_grow_kernel<QUAPI_FP64><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size);
    else if (form == QUAPI_FP32)
        herm3_grow_kernel<QUAPI_FP32><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size);
    else if (form == QUAPI_DF64)
        herm3_grow_kernel<QUAPI_DF64><<<(unsigned)blocks, kThreads, 0, st>>>(A_in, A_out, n_in, lo, hi, lo_size);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
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
    else if (M == 2 && form == QUAPI_DF64) QUAPI_GROW(2, QUAPI_DF64);
    else if (M == 3 && form == QUAPI_DF64) QUAPI_GROW(3, QUAPI_DF64);
    else return cudaErrorInvalidValue;
#undef QUAPI_GROW
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rho_reduce(const double2* partial, int nparts, int M2, double2* rho_out, cudaStream_t st) {
    if (M2 < 1 || M2 > 9) return cudaErrorInvalidValue;
    rho_reduce_kernel<<<1, kReduceLanes * M2, 0, st>>>(partial, nparts, M2, rho_out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace quapi
