// Internal declarations shared by the translation units of libquapi.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "quapi.h"

namespace quapi {

constexpr int kMaxDigits = 16;      // L <= 16 for M = 2 (4^16 entries), L <= 10 for M = 3
constexpr int kThreads = 256;       // threads per CTA of the step / growth kernels

// ---------------------------------------------------------------------------
// Complex helpers (FP64 and FP32) and double-float ("hi + lo") table entries.
// ---------------------------------------------------------------------------
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Table entry of the FP32 form: the FP64 value v split as hi = RN32(v), lo = RN32(v - hi),
// stored {hi.re, hi.im, lo.re, lo.im}.
struct __align__(16) ff2 {
    float hr, hi, lr, li;
};

// Exact sum of two floats: s + e == a + b (Knuth's TwoSum, no branch).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (T.hi + T.lo) * v for an FP32 complex v, rounded once at the end; the small
// terms are accumulated first.
__device__ __forceinline__ float2 ffmul(const ff2& T, float2 v) {
    float re = fmaf(T.lr, v.x, -T.li * v.y);
    float im = fmaf(T.lr, v.y, T.li * v.x);
    re = fmaf(T.hr, v.x, fmaf(-T.hi, v.y, re));
    im = fmaf(T.hr, v.y, fmaf(T.hi, v.x, im));
    return make_float2(re, im);
}

// T * v with the table's hi float alone: one rounded FP32 complex product.  The summed-index sums of
// the FP32 form take their products this way on the fast path, where K sits in the hi table and no
// summed-index entry carries it (its lo float would only refine a factor close to 1 below the rounding
// of the stored FP32 data; K's own rounding would leak trace, so K's tables keep both floats).
__device__ __forceinline__ float2 fmul_hi(const ff2& T, float2 v) {
    return make_float2(fmaf(T.hr, v.x, -T.hi * v.y), fmaf(T.hr, v.y, T.hi * v.x));
}

// (T.hi + T.lo) * (s + c) where (s, c) is a compensated FP32 value (|c| << |s|).
__device__ __forceinline__ float2 ffmul2(const ff2& T, float2 s, float2 c) {
    float re = fmaf(T.lr, s.x, -T.li * s.y);
    float im = fmaf(T.lr, s.y, T.li * s.x);
    re = fmaf(T.hr, c.x, fmaf(-T.hi, c.y, re));
    im = fmaf(T.hr, c.y, fmaf(T.hi, c.x, im));
    re = fmaf(T.hr, s.x, fmaf(-T.hi, s.y, re));
    im = fmaf(T.hr, s.y, fmaf(T.hi, s.x, im));
    return make_float2(re, im);
}

// Compensated complex accumulator for long sums (TwoSum on each part; the
// errors are collected in c, value = s + c).
struct cacc32 {
    float2 s, c;
    __device__ __forceinline__ void init(float2 v) { s = v; c = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float2 v) {
        float sx, ex, sy, ey;
        two_sum(s.x, v.x, sx, ex);
        two_sum(s.y, v.y, sy, ey);
        s = make_float2(sx, sy);
        c.x += ex;
        c.y += ey;
    }
    __device__ __forceinline__ void add_real(float x) {  // + x (real)
        float sx, ex;
        two_sum(s.x, x, sx, ex);
        s.x = sx;
        c.x += ex;
    }
};

// Kahan-compensated complex sum for the short sums over the summed path index
// (4 or 9 terms): value = s + c, with c the negated running correction.
struct kahan32 {
    float2 s, c;
    __device__ __forceinline__ void init(float2 v) { s = v; c = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float2 v) {
        float yx = v.x + c.x, yy = v.y + c.y;
        float tx = s.x + yx, ty = s.y + yy;
        c.x = yx - (tx - s.x);
        c.y = yy - (ty - s.y);
        s = make_float2(tx, ty);
    }
};

// ---------------------------------------------------------------------------
// Double-float form (QUAPI_DF64): a complex entry is two complex floats whose
// sum carries ~48 significant bits per component; tables are triple floats
// (t1 + t2 + t3 holds the FP64 master value exactly).  All arithmetic runs on
// the FP32 pipes with error-free transformations (TwoProd by FMA, TwoSum).
// ---------------------------------------------------------------------------
struct __align__(16) df2 {
    float2 h, l;  // value = h + l per component
};
struct __align__(16) tf2 {
    float2 t1, t2, t3, pad;
};

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}

// one real component of T * x:  T.t1 x.h exactly (TwoProd) plus the small cross terms
__device__ __forceinline__ void tf_dot_part(float t1, float t2, float t3, float xh, float xl, float& p, float& e) {
    p = t1 * xh;
    e = fmaf(t1, xh, -p);
    e = fmaf(t1, xl, e);
    e = fmaf(t2, xh, e);
    e = fmaf(t2, xl, e);
    e = fmaf(t3, xh, e);
}

// (p1 + e1) - (p2 + e2) renormalised to a double-float
__device__ __forceinline__ void df_diff(float p1, float e1, float p2, float e2, float& h, float& l) {
    float s, t;
    two_sum(p1, -p2, s, t);
    t += e1 - e2;
    fast_two_sum(s, t, h, l);
}
__device__ __forceinline__ void df_sum2(float p1, float e1, float p2, float e2, float& h, float& l) {
    float s, t;
    two_sum(p1, p2, s, t);
    t += e1 + e2;
    fast_two_sum(s, t, h, l);
}

// T * x for a triple-float table entry T and a double-float complex x
__device__ __forceinline__ df2 tfmul(const tf2& T, const df2& x) {
    float pa, ea, pb, eb, pc, ec, pd, ed;
    tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.x, x.l.x, pa, ea);  // Tre * xre
    tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.y, x.l.y, pb, eb);  // Tim * xim
    tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.y, x.l.y, pc, ec);  // Tre * xim
    tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.x, x.l.x, pd, ed);  // Tim * xre
    df2 r;
    df_diff(pa, ea, pb, eb, r.h.x, r.l.x);
    df_sum2(pc, ec, pd, ed, r.h.y, r.l.y);
    return r;
}

// Running double-float complex sum whose high parts are added with TwoSum and whose low-order
// terms are collected in plain floats; renormalised once by value().  Adding an exact product
// (high p, low-order terms e) costs two TwoSums per part instead of a renormalised product
// followed by a renormalised addition.
struct dfacc {
    float sr, er, si, ei;
    __device__ __forceinline__ void init() { sr = er = si = ei = 0.f; }
    __device__ __forceinline__ void add_hl(float ph, float pl, float qh, float ql) {  // + (ph + pl) + i (qh + ql)
        float t;
        two_sum(sr, ph, sr, t);
        er += t + pl;
        two_sum(si, qh, si, t);
        ei += t + ql;
    }
    // + T * x for a triple-float table entry T and a double-float complex x
    __device__ __forceinline__ void add_prod(const tf2& T, const df2& x) {
        float pa, ea, pb, eb, pc, ec, pd, ed, t;
        tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.x, x.l.x, pa, ea);  // Tre * xre
        tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.y, x.l.y, pb, eb);  // Tim * xim
        tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.y, x.l.y, pc, ec);  // Tre * xim
        tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.x, x.l.x, pd, ed);  // Tim * xre
        two_sum(sr, pa, sr, t);
        er += t + ea;
        two_sum(sr, -pb, sr, t);
        er += t - eb;
        two_sum(si, pc, si, t);
        ei += t + ec;
        two_sum(si, pd, si, t);
        ei += t + ed;
    }
    __device__ __forceinline__ df2 value() const {
        df2 r;
        fast_two_sum(sr, er, r.h.x, r.l.x);
        fast_two_sum(si, ei, r.h.y, r.l.y);
        return r;
    }
    // Starting from the first term instead of adding it to zero (IEEE arithmetic keeps the
    // compiler from dropping a TwoSum with 0):  = (ph + pl) + i (qh + ql)
    __device__ __forceinline__ void init_hl(float ph, float pl, float qh, float ql) {
        sr = ph;
        er = pl;
        si = qh;
        ei = ql;
    }
    //  = T * x
    __device__ __forceinline__ void init_prod(const tf2& T, const df2& x) {
        float pb, eb, pd, ed, t;
        tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.x, x.l.x, sr, er);  // Tre * xre
        tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.y, x.l.y, pb, eb);  // Tim * xim
        tf_dot_part(T.t1.x, T.t2.x, T.t3.x, x.h.y, x.l.y, si, ei);  // Tre * xim
        tf_dot_part(T.t1.y, T.t2.y, T.t3.y, x.h.x, x.l.x, pd, ed);  // Tim * xre
        two_sum(sr, -pb, sr, t);
        er += t - eb;
        two_sum(si, pd, si, t);
        ei += t + ed;
    }
    // The unrenormalised pair (sr + er) + i (si + ei), for a value that is only multiplied next:
    // a product takes the pair's two parts as they are (TwoProd of the high part, the low part's
    // products added to the error term), so renormalising first would not change its accuracy.
    __device__ __forceinline__ df2 raw() const {
        df2 r;
        r.h = make_float2(sr, si);
        r.l = make_float2(er, ei);
        return r;
    }
};

// x + y for double-float complex values (TwoSum on the high parts)
__device__ __forceinline__ df2 dfadd(const df2& x, const df2& y) {
    df2 r;
    float s, t;
    two_sum(x.h.x, y.h.x, s, t);
    t += x.l.x + y.l.x;
    fast_two_sum(s, t, r.h.x, r.l.x);
    two_sum(x.h.y, y.h.y, s, t);
    t += x.l.y + y.l.y;
    fast_two_sum(s, t, r.h.y, r.l.y);
    return r;
}

// ---------------------------------------------------------------------------
// Host-side description of one tensor operation (growth, step or readout).
// ---------------------------------------------------------------------------
enum OpKind { OP_GROW = 0, OP_STEP = 1, OP_READ = 2 };

struct OpPlan {
    int kind = OP_STEP;
    int n_in = 0;        // digits of the input tensor
    int summed = 0;      // 1 if digit 0 is summed (step, readout)
    int nk = 0;          // kept digits (n_in - summed)
    int j = 0;           // kept digits resolved by the lo table
    int64_t lo_size = 1; // (M^2)^j
    int64_t hi_size = 1; // (M^2)^(nk - j)
    int eta_idx[kMaxDigits] = {0};  // eta index (into the 4L+3 vector) per input digit
    int self_idx = 0;    // eta index of the new point's self term
    size_t off_isum = 0, off_lo = 0, off_hi = 0;  // byte offsets in the table arena
    size_t off_w = 0;    // summed ops: w[x][f_lo][old] = lo[x][f_lo] * isum[x][old]
};

// Device-side build request for one OpPlan (all pointers device).
struct BuildDesc {
    int M, M2, n_in, summed, nk, j, form;   // form: 64 or 32
    int eta_idx[kMaxDigits];
    int self_idx;
    int64_t lo_size, hi_size;
    const double2* eta;
    const double* s;
    const double2* K;
    void* isum;
    void* lo;
    void* hi;
    void* w;              // summed ops: lo (x) isum, M2 x lo_size x M2 entries
};

// eta quadrature request: one integral per entry.
struct EtaJob {
    double w1, w2, D;   // box widths (later, earlier) and centre distance; w2 < 0 marks a self box
};

// ---------------------------------------------------------------------------
// Launchers implemented in the .cu files.
// ---------------------------------------------------------------------------
cudaError_t launch_eta_quadrature(const EtaJob* jobs_dev, int njobs, int kind, double a, double wc,
                                  double beta, int panels, const double* gl_dev, int gl_n,
                                  double2* eta_out, cudaStream_t st);
// tabulated J: panel end points pw[0..panels] and J at them pj[0..panels] (J linear on each panel)
cudaError_t launch_eta_quadrature_tab(const EtaJob* jobs_dev, int njobs, double beta, const double* pw_dev,
                                      const double* pj_dev, int panels, const double* gl_dev, int gl_n,
                                      double2* eta_out, cudaStream_t st);
void gauss_legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w);

cudaError_t launch_propagator(const double2* H_dev, int M, double dt, double2* U_dev, double2* K_dev,
                              cudaStream_t st);
cudaError_t launch_build_tables(const BuildDesc* descs_dev, int ndesc, int M2, int64_t max_entries,
                                cudaStream_t st);

struct StepArgs {
    const void* A_in;
    void* A_out;          // may be null (readout only)
    int64_t F;            // input fibers = (M^2)^(n_in - 1)
    const void* isum;     // step tables
    const void* lo;
    const void* hi;
    const void* isum_e;   // readout tables (null if no readout)
    const void* lo_e;
    const void* hi_e;
    const void* w;        // lo (x) isum of the step, [x][f_lo][old]
    const void* w_e;      // the same for the readout
    int64_t lo_size;      // (M^2)^j, common to step and readout tables
    int lo_shift;         // log2(lo_size) when M = 2
    double2* partial;     // [grid][M^2] readout partial sums
    int grid;             // in: upper bound (partial buffer size); out: CTAs launched
    bool diag_fast;
    bool use_tma;         // M = 2: stage input tiles with 2-D TMA copies when the tensor allows it
    int stages;           // TMA ring depth (2, 3, 4 or 6)
    int* err_flag;        // set to 1 by a CTA whose bounded wait expired
    int half_digits;      // Hermitian half layout (M = 2 or 3): digits of the fiber prefix (n_in - 1)
    int eq_spaced;        // M = 3: equally spaced s (rows with equal s_a - s_b share isum and lo rows)
    uint64_t wait_ns;     // limit of every device-side wait (QUAPI_WAIT_MS at set-up; default 2 s)
    uint32_t fault_tx;    // host-side fault injection (QUAPI_FAULT=tma_tx at set-up): bytes added to the
                          // first tile's expected transfer in CTA 0 of the TMA step, so that its wait expires
};

cudaError_t launch_step(int M, int form, StepArgs& a, cudaStream_t st);  // sets a.grid
cudaError_t launch_grow(int M, int form, const void* A_in, void* A_out, int64_t S, const void* lo,
                        const void* hi, int64_t lo_size, int lo_shift, cudaStream_t st);
cudaError_t launch_herm_step(int form, StepArgs& a, cudaStream_t st);  // sets a.grid
cudaError_t launch_herm_grow(int form, const void* A_in, void* A_out, int n_in, const void* lo, const void* hi,
                             int64_t lo_size, int lo_shift, cudaStream_t st);
cudaError_t launch_herm3_step(int form, StepArgs& a, cudaStream_t st);  // M = 3 half layout; sets a.grid
cudaError_t launch_herm3_grow(int form, const void* A_in, void* A_out, int n_in, const void* lo, const void* hi,
                              int64_t lo_size, cudaStream_t st);
cudaError_t launch_rho_reduce(const double2* partial, int nparts, int M2, double2* rho_out,
                              cudaStream_t st);
cudaError_t launch_init_tensor(const double2* rho0_dev, const double2* eta, int self0_idx,
                               const double* s, int M, int form, void* A_out, cudaStream_t st, int herm = 0);
int num_sms();

// process-wide count of kernel launches issued by this library
void count_launch(uint64_t n = 1);
uint64_t launches_so_far();

}  // namespace quapi

struct quapi_ctx;
namespace quapi {
quapi_status readout_launch_args(const ::quapi_ctx* c, int64_t n, const void* A_in, StepArgs* a, int* M,
                                 int* form, cudaStream_t* st);
quapi_status record_error(const ::quapi_ctx* c, quapi_status st, const char* msg);
}  // namespace quapi

namespace quapi {

// One operation's tables inside a context's arena (device pointers).
struct OpRef {
    const void* isum = nullptr;
    const void* lo = nullptr;
    const void* hi = nullptr;
    int64_t lo_size = 1;
    int lo_shift = 0;
    int64_t hi_size = 1;
    int n_in = 0;
    int diag = 0;  // diagonal fast path valid for this operation
};

// Everything the batched kernel needs about one instance (device-visible copy).
struct BatchInst {
    void* buf[2];
    int L, N, resident;
    int herm;                // tensors in the Hermitian half layout (M = 2)
    int self0_idx;
    const double2* eta;
    const double* s;
    OpRef grow[kMaxDigits];  // growth step n = 1..L-1 at index n
    OpRef step_first;        // n == L
    OpRef step;              // n > L
    OpRef read;              // readout at n == N
    double2* partial;        // [readout tiles][M^2]
    unsigned int* done;      // tiles completed over all steps
    unsigned int* read_done; // readout tiles completed
    double2* rho_out;        // M^2 (device)
    const double2* rho0;     // M^2 (device)
};

uint64_t ctx_uid(const ::quapi_ctx* c);            // unique per context for the process lifetime
int ctx_device(const ::quapi_ctx* c);              // CUDA device that was current at the context's setup
bool ctx_tune_requested(const ::quapi_ctx* c);     // quapi_opts.tune was set
bool ctx_half_layout(const ::quapi_ctx* c);        // tensors in the Hermitian half layout
void batch_forget(uint64_t uid);                    // drop cached batch plans using that context

// Fill inst with the tables and tensors of context c for a run to step N (host side).
quapi_status batch_describe(const ::quapi_ctx* c, int64_t N, BatchInst* inst, int* M, int* form, cudaStream_t* st,
                            int* L);
}  // namespace quapi
