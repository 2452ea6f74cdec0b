// Host side of libquapi.so: argument checks, the step planner (which eta
// coefficient joins which pair of path points), device memory, and the C ABI
// entry points declared in include/quapi.h.
//
// Path bookkeeping (Sec. II, truncated influence functional; Sec. I, tensor
// propagator scheme).  The tensor A_{n-1} that feeds the step adding path
// point n holds n_in = min(n, L) points; input digit p holds point
// n - n_in + p.  The new point pairs with each stored point at distance
// dk = n - point <= L:
//   growth / step tensor (new point propagates on as an interior point):
//     point 0 -> eta_{n0} (Eq. etaK0generalStrang), otherwise interior eta_dk,
//     self term interior eta_0;
//   readout of rho(t_n) (STRANG end point, Eqs. etaNNgeneralStrang,
//   etaNkgeneralStrang, etaN0generalStrang):
//     point 0 -> eta_{n0}^{end}, otherwise eta_{n,n-dk}^{end}, self eta_NN.
// Once n >= L the oldest stored point is summed (it leaves the memory window).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "quapi_internal.h"

using namespace quapi;

namespace quapi {
static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace quapi

namespace {

thread_local std::string g_thread_error;

// indices into the 4L+3 eta vector (layout documented in quapi.h)
inline int eta_interior(int L, int dk) { (void)L; return dk; }
inline int eta_point0(int L, int k) { return L + 1 + (k - 1); }
inline int eta_end_self(int L) { return 2 * L + 1; }
inline int eta_end(int L, int dk) { return 2 * L + 2 + (dk - 1); }
inline int eta_end_point0(int L, int N) { return 3 * L + 2 + (N - 1); }
inline int eta_self0(int L) { return 4 * L + 2; }

int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

int max_dkmax(int M) { return M == 2 ? 16 : 10; }
constexpr int kMaxTableNodes = 65536;          // tabulated J: largest table
constexpr int64_t kMaxEtaPanels = int64_t(1) << 22;  // tabulated J: largest panel count

// stored entries of an n-digit tensor in the Hermitian half layout: M^2 C(n-1), C(m) = ((M^2)^m + M^m)/2
int64_t half_entries(int M, int n) {
    if (n == 0) return 1;
    return (int64_t)M * M * ((ipow((int64_t)M * M, n - 1) + ipow(M, n - 1)) >> 1);
}
int lo_digits_max(int M) { return M == 2 ? 4 : 2; }

}  // namespace

struct quapi_ctx {
    int M = 0, M2 = 0, L = 0, form = QUAPI_FP64, endpoint = QUAPI_ENDPOINT_STRANG;
    double dt = 0.0;
    cudaStream_t st = nullptr;
    double* d_s = nullptr;
    double2 *d_H = nullptr, *d_U = nullptr, *d_K = nullptr, *d_eta = nullptr, *d_rho0 = nullptr;
    double2* d_slots = nullptr;
    size_t slots_cap = 0;
    void* buf[2] = {nullptr, nullptr};
    bool own_buf = true;
    unsigned char* d_tables = nullptr;
    double2* d_partial = nullptr;
    int* d_err = nullptr;        // set by a kernel whose bounded wait expired
    int max_grid = 0;
    bool use_tma = true;         // M = 2: TMA-staged step kernel when the tensor allows it
    int stages = 2;              // its ring depth (2 measured best: 4 CTAs per SM fit)
    bool tune = false;           // quapi_opts.tune
    bool herm = false;           // Hermitian half layout (M = 2 or 3)
    int64_t state_n = -1;        // path point of the newest tensor kept in buf[state_buf] (-1: none)
    int state_buf = 0;
    uint64_t uid = 0;            // never reused within the process
    int device = -1;             // CUDA device current at setup (its memory holds the context's tables)
    int eq_spaced = 0;           // M = 3 with s_1 - s_0 = s_2 - s_1 (exactly, in FP64)
    uint64_t wait_ns = 2000000000ull;  // limit of the step kernels' device-side waits
    uint32_t fault_tx = 0;       // host-side fault injection into the TMA step (testing)
    // A whole propagation captured as a CUDA graph and replayed when the same call (rho0 buffer, rho
    // slots, step list) comes again: one graph launch instead of one host launch sequence per step
    // (which bounds small, L2-resident tensors).  The first call with new arguments runs directly and
    // only records them; the second captures on a private stream and replays from then on.
    struct PropGraph {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;     // the capture stream (non-blocking, created on first use)
        bool ready = false;             // exec holds the propagation of the recorded arguments
        const void* rho0 = nullptr;
        const void* slots = nullptr;
        std::vector<int64_t> steps;
        int64_t state_n = -1;           // the host bookkeeping the captured propagation leaves
        int state_buf = 0;
        uint64_t launches = 0;          // kernels in the graph
    } graph;
    bool graphs = true;             // QUAPI_GRAPH=0 turns the replay off
    std::vector<OpPlan> grow_ops;   // index n = 1..L-1
    std::vector<OpPlan> read_ops;   // index N = 1..L
    OpPlan step_first, step_steady, read_steady;
    std::string err;
    std::vector<double> host_s;
};

namespace {

quapi_status fail(quapi_ctx* c, quapi_status st, const std::string& msg) {
    if (c) c->err = msg;
    g_thread_error = msg;
    return st;
}

quapi_status cuda_fail(quapi_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? QUAPI_ERR_OOM : QUAPI_ERR_CUDA, m);
}

#define QCHECK(c, call, what)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, (what)); \
    } while (0)

size_t elem_bytes(int form) { return form == QUAPI_FP32 ? 8 : 16; }
size_t table_entry_bytes(int form) { return form == QUAPI_DF64 ? 32 : 16; }
bool valid_precision(int p) { return p == QUAPI_FP64 || p == QUAPI_FP32 || p == QUAPI_DF64; }

// Plan of one operation on an input tensor of n_in digits.
OpPlan make_plan(int M, int kind, int n_in, bool summed, const int* eta_idx, int self_idx) {
    OpPlan p;
    p.kind = kind;
    p.n_in = n_in;
    p.summed = summed ? 1 : 0;
    p.nk = n_in - p.summed;
    p.j = std::min(p.nk, lo_digits_max(M));
    p.lo_size = ipow(M * M, p.j);
    p.hi_size = ipow(M * M, p.nk - p.j);
    for (int q = 0; q < n_in; ++q) p.eta_idx[q] = eta_idx[q];
    p.self_idx = self_idx;
    return p;
}

OpPlan plan_step(int M, int L, int64_t n) {
    int n_in = (int)std::min<int64_t>(n, L);
    int idx[kMaxDigits];
    for (int p = 0; p < n_in; ++p) {
        int64_t point = n - n_in + p;
        int dk = (int)(n - point);
        idx[p] = (point == 0) ? eta_point0(L, (int)n) : eta_interior(L, dk);
    }
    bool summed = n >= L;
    return make_plan(M, summed ? OP_STEP : OP_GROW, n_in, summed, idx, eta_interior(L, 0));
}

OpPlan plan_readout(int M, int L, int64_t N, int endpoint) {
    int n_in = (int)std::min<int64_t>(N, L);
    int idx[kMaxDigits];
    for (int p = 0; p < n_in; ++p) {
        int64_t point = N - n_in + p;
        int dk = (int)(N - point);
        if (endpoint == QUAPI_ENDPOINT_STRANG)
            idx[p] = (point == 0) ? eta_end_point0(L, (int)N) : eta_end(L, dk);
        else
            idx[p] = (point == 0) ? eta_point0(L, (int)N) : eta_interior(L, dk);
    }
    int self = endpoint == QUAPI_ENDPOINT_STRANG ? eta_end_self(L) : eta_interior(L, 0);
    return make_plan(M, OP_READ, n_in, true, idx, self);
}

void assign_offsets(OpPlan& p, int M2, int form, size_t& cursor) {
    const size_t e = table_entry_bytes(form);
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    cursor = align(cursor);
    p.off_isum = cursor;
    if (p.summed) cursor += (size_t)M2 * M2 * e;
    cursor = align(cursor);
    p.off_lo = cursor;
    cursor += (size_t)M2 * p.lo_size * e;
    cursor = align(cursor);
    p.off_hi = cursor;
    cursor += (size_t)M2 * p.hi_size * e;
    cursor = align(cursor);
    p.off_w = cursor;
    if (p.summed) cursor += (size_t)M2 * p.lo_size * M2 * e;
}

// every table set the context needs, in a fixed order
std::vector<OpPlan*> all_plans(quapi_ctx* c) {
    std::vector<OpPlan*> v;
    for (int n = 1; n < c->L; ++n) v.push_back(&c->grow_ops[n]);
    for (int N = 1; N <= c->L; ++N) v.push_back(&c->read_ops[N]);
    v.push_back(&c->step_first);
    v.push_back(&c->step_steady);
    v.push_back(&c->read_steady);
    return v;
}

void make_all_plans(quapi_ctx* c) {
    c->grow_ops.assign(c->L + 1, OpPlan());
    c->read_ops.assign(c->L + 1, OpPlan());
    for (int n = 1; n < c->L; ++n) c->grow_ops[n] = plan_step(c->M, c->L, n);
    for (int N = 1; N <= c->L; ++N) c->read_ops[N] = plan_readout(c->M, c->L, N, c->endpoint);
    c->step_first = plan_step(c->M, c->L, c->L);
    c->step_steady = plan_step(c->M, c->L, c->L + 1);
    c->read_steady = plan_readout(c->M, c->L, c->L + 1, c->endpoint);
}

size_t tables_bytes_for(int M, int L, int endpoint, int form) {
    quapi_ctx tmp;
    tmp.M = M;
    tmp.M2 = M * M;
    tmp.L = L;
    tmp.endpoint = endpoint;
    make_all_plans(&tmp);
    size_t cursor = 0;
    for (OpPlan* p : all_plans(&tmp)) assign_offsets(*p, tmp.M2, form, cursor);
    return cursor + 256;
}

quapi_status check_common(const double* s, int M, const double* H, double dt, int L, const quapi_opts* o) {
    if (!s || !H) return fail(nullptr, QUAPI_ERR_ARG, "s and H must not be NULL");
    if (M != 2 && M != 3) return fail(nullptr, QUAPI_ERR_ARG, "M must be 2 or 3");
    if (L < 1 || L > max_dkmax(M)) return fail(nullptr, QUAPI_ERR_ARG, "dkmax out of range (1..16 for M=2, 1..10 for M=3)");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, QUAPI_ERR_ARG, "dt must be > 0");
    for (int i = 0; i < M; ++i)
        if (!std::isfinite(s[i])) return fail(nullptr, QUAPI_ERR_ARG, "s must be finite");
    for (int r = 0; r < M; ++r)
        for (int q = 0; q < M; ++q) {
            double ar = H[2 * (r * M + q)], ai = H[2 * (r * M + q) + 1];
            double br = H[2 * (q * M + r)], bi = H[2 * (q * M + r) + 1];
            if (!std::isfinite(ar) || !std::isfinite(ai)) return fail(nullptr, QUAPI_ERR_ARG, "H must be finite");
            if (std::fabs(ar - br) > 1e-12 || std::fabs(ai + bi) > 1e-12)
                return fail(nullptr, QUAPI_ERR_ARG, "H must be Hermitian (tolerance 1e-12)");
        }
    if (o) {
        if (!valid_precision(o->precision))
            return fail(nullptr, QUAPI_ERR_ARG, "precision must be QUAPI_FP64, QUAPI_FP32 or QUAPI_DF64");
        if (o->endpoint_mode != QUAPI_ENDPOINT_STRANG && o->endpoint_mode != QUAPI_ENDPOINT_INTERIOR)
            return fail(nullptr, QUAPI_ERR_ARG, "unknown endpoint_mode");
    }
    return QUAPI_OK;
}

quapi_status tune_step(quapi_ctx* c);

// Caller device buffers: the kernels read and write them with 16-byte vector accesses and bulk
// copies (NULL passes; it is checked separately).
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Device buffers a function needs only while it runs: freed when it returns, on every path.
struct DeviceScratch {
    std::vector<void*> ptrs;
    template <class T> cudaError_t alloc(T** p, size_t bytes) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~DeviceScratch() {
        for (void* q : ptrs) cudaFree(q);
    }
};

// Allocation, eta (given or by quadrature), propagators and tables.
quapi_status setup_impl(const double* s, int M, const double* H, const quapi_spectral* J, double beta,
                        const double* eta_host, double dt, int L, const quapi_opts* opts, quapi_ctx** out) {
    if (!out) return fail(nullptr, QUAPI_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    quapi_opts o;
    quapi_opts_init(&o);
    if (opts) o = *opts;
    quapi_status stc = check_common(s, M, H, dt, L, &o);
    if (stc != QUAPI_OK) return stc;
    if (!eta_host) {
        if (!J) return fail(nullptr, QUAPI_ERR_ARG, "J must not be NULL");
        if (J->kind == QUAPI_J_TABULATED) {
            if (!J->omega || !J->values || J->n < 1 || J->n > kMaxTableNodes)
                return fail(nullptr, QUAPI_ERR_ARG, "tabulated J needs 1..65536 nodes and non-NULL arrays");
            for (int i = 0; i < J->n; ++i) {
                const double w = J->omega[i], v = J->values[i];
                if (!std::isfinite(w) || !std::isfinite(v) || v < 0.0 || w <= (i ? J->omega[i - 1] : 0.0))
                    return fail(nullptr, QUAPI_ERR_ARG,
                                "tabulated J needs finite, strictly ascending omega > 0 and finite values >= 0");
            }
        } else if (J->kind == QUAPI_J_OHMIC_EXP || J->kind == QUAPI_J_SUPEROHMIC_GAUSS) {
            if (!(J->a >= 0.0) || !(J->wc > 0.0) || !std::isfinite(J->a) || !std::isfinite(J->wc))
                return fail(nullptr, QUAPI_ERR_ARG, "spectral density needs a >= 0 and wc > 0");
        } else {
            return fail(nullptr, QUAPI_ERR_ARG, "unknown spectral density kind");
        }
        if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, QUAPI_ERR_ARG, "beta must be > 0");
    }
    const int M2 = M * M;
    const int64_t nelem = o.hermitian ? half_entries(M, L) : ipow(M2, L);
    const size_t tensor_bytes = 2 * (size_t)nelem * elem_bytes(o.precision);
    if (o.workspace && o.workspace_bytes < tensor_bytes)
        return fail(nullptr, QUAPI_ERR_OOM, "caller workspace smaller than the two tensors");
    if (!aligned16(o.workspace)) return fail(nullptr, QUAPI_ERR_ARG, "caller workspace must be 16-byte aligned");

    quapi_ctx* c = new quapi_ctx();
    c->M = M;
    c->M2 = M2;
    c->L = L;
    c->dt = dt;
    c->form = o.precision;
    c->endpoint = o.endpoint_mode;
    c->st = reinterpret_cast<cudaStream_t>(o.cuda_stream);
    c->host_s.assign(s, s + M);
    // d(x) = s_a - s_b computed the same way as the table kernel: equal values give bitwise equal rows
    c->eq_spaced = (M == 3 && (s[0] - s[1]) == (s[1] - s[2])) ? 1 : 0;
    cudaGetDevice(&c->device);
    c->tune = o.tune != 0;
    c->herm = o.hermitian != 0;
    {
        static std::atomic<uint64_t> next_uid{1};
        c->uid = next_uid.fetch_add(1);
    }
    auto bail = [&](quapi_status st) {
        std::string m = c->err;
        quapi_destroy(c);
        g_thread_error = m;
        return st;
    };
#define SCHECK(call, what)                                            \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, (what))); \
    } while (0)

    const int neta = 4 * L + 3;
    SCHECK(cudaMalloc(&c->d_s, sizeof(double) * M), "cudaMalloc(s)");
    SCHECK(cudaMalloc(&c->d_H, sizeof(double2) * M * M), "cudaMalloc(H)");
    SCHECK(cudaMalloc(&c->d_U, sizeof(double2) * M * M), "cudaMalloc(U)");
    SCHECK(cudaMalloc(&c->d_K, sizeof(double2) * M2 * M2), "cudaMalloc(K)");
    SCHECK(cudaMalloc(&c->d_eta, sizeof(double2) * neta), "cudaMalloc(eta)");
    SCHECK(cudaMalloc(&c->d_rho0, sizeof(double2) * M2), "cudaMalloc(rho0)");
    if (o.workspace) {
        c->own_buf = false;
        c->buf[0] = o.workspace;
        c->buf[1] = static_cast<unsigned char*>(o.workspace) + tensor_bytes / 2;
    } else {
        SCHECK(cudaMalloc(&c->buf[0], tensor_bytes / 2), "cudaMalloc(tensor A)");
        SCHECK(cudaMalloc(&c->buf[1], tensor_bytes / 2), "cudaMalloc(tensor B)");
    }
    make_all_plans(c);
    size_t cursor = 0;
    for (OpPlan* p : all_plans(c)) assign_offsets(*p, M2, c->form, cursor);
    SCHECK(cudaMalloc(&c->d_tables, cursor + 256), "cudaMalloc(tables)");
    c->max_grid = num_sms() * 8;  // at most 8 resident CTAs of 256 threads per SM
    SCHECK(cudaMalloc(&c->d_partial, sizeof(double2) * M2 * (size_t)c->max_grid), "cudaMalloc(partials)");
    SCHECK(cudaMalloc(&c->d_err, sizeof(int)), "cudaMalloc(error flag)");
    SCHECK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st), "clear error flag");
    if (const char* v = std::getenv("QUAPI_TMA")) c->use_tma = std::atoi(v) != 0;
    if (const char* v = std::getenv("QUAPI_GRAPH")) c->graphs = std::atoi(v) != 0;
    if (const char* v = std::getenv("QUAPI_WAIT_MS")) {
        const double ms = std::atof(v);
        if (ms > 0) c->wait_ns = (uint64_t)(ms * 1e6);
    }
    // host-side fault injection: CTA 0 of every TMA step expects 16 bytes more than its first tile's
    // copies deliver, so its bounded wait expires and the call reports QUAPI_ERR_TIMEOUT
    if (const char* f = std::getenv("QUAPI_FAULT"))
        if (std::strcmp(f, "tma_tx") == 0) c->fault_tx = 16;
    if (const char* v = std::getenv("QUAPI_STAGES")) {
        int k = std::atoi(v);
        if (k == 2 || k == 3 || k == 4 || k == 6) c->stages = k;
    }

    SCHECK(cudaMemcpyAsync(c->d_s, s, sizeof(double) * M, cudaMemcpyHostToDevice, c->st), "copy s");
    SCHECK(cudaMemcpyAsync(c->d_H, H, sizeof(double2) * M * M, cudaMemcpyHostToDevice, c->st), "copy H");
    SCHECK(launch_propagator(c->d_H, M, dt, c->d_U, c->d_K, c->st), "propagator kernel");

    DeviceScratch scratch;  // set-up scratch on the device, freed when set-up returns (also on errors)
    EtaJob* d_jobs = nullptr;
    double* d_gl = nullptr;
    double* d_pan = nullptr;  // tabulated J: panel end points, then J at them
    if (eta_host) {
        SCHECK(cudaMemcpyAsync(c->d_eta, eta_host, sizeof(double2) * neta, cudaMemcpyHostToDevice, c->st),
               "copy eta");
    } else {
        // box geometry of every eta (symmetric placement): point 0 owns [0, dt/2],
        // interior point k owns [(k-1/2)dt, (k+1/2)dt], the end point N owns [(N-1/2)dt, N dt]
        std::vector<EtaJob> jobs(neta);
        auto self = [](double w) { return EtaJob{w, -1.0, 0.0}; };
        auto pair = [](double w1, double w2, double D) { return EtaJob{w1, w2, D}; };
        jobs[eta_interior(L, 0)] = self(dt);
        for (int dk = 1; dk <= L; ++dk) jobs[eta_interior(L, dk)] = pair(dt, dt, dk * dt);
        for (int k = 1; k <= L; ++k) jobs[eta_point0(L, k)] = pair(dt, 0.5 * dt, k * dt - 0.25 * dt);
        jobs[eta_end_self(L)] = self(0.5 * dt);
        for (int dk = 1; dk <= L; ++dk) jobs[eta_end(L, dk)] = pair(0.5 * dt, dt, dk * dt - 0.25 * dt);
        for (int N = 1; N <= L; ++N) jobs[eta_end_point0(L, N)] = pair(0.5 * dt, 0.5 * dt, N * dt - 0.5 * dt);
        jobs[eta_self0(L)] = self(0.5 * dt);
        double kmax = 0.0;
        for (const EtaJob& jb : jobs) kmax = std::max(kmax, jb.w2 < 0 ? jb.w1 : jb.D + 0.5 * (jb.w1 + jb.w2));
        std::vector<double> gx, gw;
        gauss_legendre_nodes(16, gx, gw);
        std::vector<double> gl(gx);
        gl.insert(gl.end(), gw.begin(), gw.end());
        SCHECK(scratch.alloc(&d_jobs, sizeof(EtaJob) * neta), "cudaMalloc(eta jobs)");
        SCHECK(scratch.alloc(&d_gl, sizeof(double) * gl.size()), "cudaMalloc(GL nodes)");
        SCHECK(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(EtaJob) * neta, cudaMemcpyHostToDevice, c->st), "copy jobs");
        SCHECK(cudaMemcpyAsync(d_gl, gl.data(), sizeof(double) * gl.size(), cudaMemcpyHostToDevice, c->st), "copy GL");
        if (J->kind == QUAPI_J_TABULATED) {
            // segments (0, 0) -> (omega[0], values[0]) -> ...; each cut into panels no wider than the
            // parametric rule's (2 / kmax, at least 256 panels over [0, omega[n-1]])
            const double wmax = J->omega[J->n - 1];
            std::vector<double> pw, pj;
            double t0 = 0.0, j0 = 0.0;
            for (int k = 0; k < J->n; ++k) {
                const double t1 = J->omega[k], j1 = J->values[k], len = t1 - t0;
                const double want = std::max(len * kmax / 2.0, 256.0 * len / wmax);
                const int64_t m = std::max<int64_t>(1, (int64_t)std::ceil(want));
                if ((int64_t)pw.size() + m > kMaxEtaPanels)
                    return bail(fail(c, QUAPI_ERR_ARG, "tabulated J too wide for the eta quadrature panels"));
                for (int64_t q = 0; q < m; ++q) {
                    pw.push_back(t0 + len * (double)q / (double)m);
                    pj.push_back(j0 + (j1 - j0) * (double)q / (double)m);
                }
                t0 = t1;
                j0 = j1;
            }
            pw.push_back(t0);
            pj.push_back(j0);
            const int panels = (int)pw.size() - 1;
            pw.insert(pw.end(), pj.begin(), pj.end());
            SCHECK(scratch.alloc(&d_pan, sizeof(double) * pw.size()), "cudaMalloc(eta panels)");
            SCHECK(cudaMemcpyAsync(d_pan, pw.data(), sizeof(double) * pw.size(), cudaMemcpyHostToDevice, c->st),
                   "copy eta panels");
            SCHECK(launch_eta_quadrature_tab(d_jobs, neta, beta, d_pan, d_pan + panels + 1, panels, d_gl, 16,
                                             c->d_eta, c->st),
                   "eta quadrature kernel (tabulated J)");
            SCHECK(cudaStreamSynchronize(c->st), "eta quadrature (tabulated J)");  // pw leaves scope
        } else {
            const double wmax = (J->kind == QUAPI_J_OHMIC_EXP) ? 46.0 * J->wc : 7.5 * J->wc;
            int panels = (int)std::ceil(wmax * kmax / 2.0);
            panels = std::max(panels, 256);
            panels = std::min(panels, 1 << 16);
            SCHECK(launch_eta_quadrature(d_jobs, neta, J->kind, J->a, J->wc, beta, panels, d_gl, 16, c->d_eta,
                                         c->st),
                   "eta quadrature kernel");
        }
    }

    // factor tables of every operation, one launch
    std::vector<OpPlan*> plans = all_plans(c);
    std::vector<BuildDesc> descs(plans.size());
    int64_t max_entries = 0;
    for (size_t i = 0; i < plans.size(); ++i) {
        const OpPlan& p = *plans[i];
        BuildDesc& d = descs[i];
        std::memset(&d, 0, sizeof(d));
        d.M = M;
        d.M2 = M2;
        d.n_in = p.n_in;
        d.summed = p.summed;
        d.nk = p.nk;
        d.j = p.j;
        d.form = c->form;
        for (int q = 0; q < p.n_in; ++q) d.eta_idx[q] = p.eta_idx[q];
        d.self_idx = p.self_idx;
        d.lo_size = p.lo_size;
        d.hi_size = p.hi_size;
        d.eta = c->d_eta;
        d.s = c->d_s;
        d.K = c->d_K;
        d.isum = c->d_tables + p.off_isum;
        d.lo = c->d_tables + p.off_lo;
        d.hi = c->d_tables + p.off_hi;
        d.w = c->d_tables + p.off_w;
        int64_t ent = (p.summed ? M2 * M2 + M2 * p.lo_size * M2 : 0) + M2 * p.lo_size + M2 * p.hi_size;
        max_entries = std::max(max_entries, ent);
    }
    BuildDesc* d_descs = nullptr;
    SCHECK(scratch.alloc(&d_descs, sizeof(BuildDesc) * descs.size()), "cudaMalloc(build descs)");
    SCHECK(cudaMemcpyAsync(d_descs, descs.data(), sizeof(BuildDesc) * descs.size(), cudaMemcpyHostToDevice, c->st),
           "copy build descs");
    SCHECK(launch_build_tables(d_descs, (int)descs.size(), M2, max_entries, c->st), "table build kernel");
    SCHECK(cudaStreamSynchronize(c->st), "setup synchronize");
    if (c->tune) {
        quapi_status ts = tune_step(c);
        if (ts != QUAPI_OK) return bail(ts);
    }
#undef SCHECK
    *out = c;
    return QUAPI_OK;
}

// Readout on A_in (n_in digits) with plan rp, optionally fused with the step plan sp.
quapi_status run_step_op(quapi_ctx* c, const OpPlan* sp, const OpPlan* rp, const void* A_in, void* A_out,
                         double2* rho_slot) {
    const int64_t F = ipow(c->M2, (sp ? sp->n_in : rp->n_in) - 1);
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.A_in = A_in;
    a.A_out = A_out;
    a.F = F;
    const OpPlan* ref = sp ? sp : rp;
    if (sp) {
        a.isum = c->d_tables + sp->off_isum;
        a.lo = c->d_tables + sp->off_lo;
        a.hi = c->d_tables + sp->off_hi;
        a.w = c->d_tables + sp->off_w;
    }
    if (rp) {
        a.isum_e = c->d_tables + rp->off_isum;
        a.lo_e = c->d_tables + rp->off_lo;
        a.hi_e = c->d_tables + rp->off_hi;
        a.w_e = c->d_tables + rp->off_w;
        a.partial = c->d_partial;
    }
    a.lo_size = ref->lo_size;
    int sh = 0;
    while ((int64_t(1) << sh) < ref->lo_size) ++sh;
    a.lo_shift = sh;
    a.grid = c->max_grid;
    a.diag_fast = ref->n_in >= 2 && ref->nk > ref->j;
    a.use_tma = c->use_tma;
    a.stages = c->stages;
    a.err_flag = c->d_err;
    a.eq_spaced = c->eq_spaced;
    a.wait_ns = c->wait_ns;
    a.fault_tx = c->fault_tx;
    a.half_digits = c->herm ? ref->n_in - 1 : -1;
    if (c->herm && c->M == 3)
        QCHECK(c, launch_herm3_step(c->form, a, c->st), "half-layout step kernel");
    else if (c->herm)
        QCHECK(c, launch_herm_step(c->form, a, c->st), "half-layout step kernel");
    else
        QCHECK(c, launch_step(c->M, c->form, a, c->st), "step kernel");
    if (rp) QCHECK(c, launch_rho_reduce(c->d_partial, a.grid, c->M2, rho_slot, c->st), "rho reduce kernel");
    return QUAPI_OK;
}

quapi_status run_grow_op(quapi_ctx* c, const OpPlan& gp, const void* A_in, void* A_out) {
    int sh = 0;
    while ((int64_t(1) << sh) < gp.lo_size) ++sh;
    if (c->herm && c->M == 3) {
        QCHECK(c, launch_herm3_grow(c->form, A_in, A_out, gp.n_in, c->d_tables + gp.off_lo, c->d_tables + gp.off_hi,
                                    gp.lo_size, c->st),
               "half-layout grow kernel");
        return QUAPI_OK;
    }
    if (c->herm) {
        QCHECK(c, launch_herm_grow(c->form, A_in, A_out, gp.n_in, c->d_tables + gp.off_lo, c->d_tables + gp.off_hi,
                                   gp.lo_size, sh, c->st),
               "half-layout grow kernel");
        return QUAPI_OK;
    }
    QCHECK(c, launch_grow(c->M, c->form, A_in, A_out, ipow(c->M2, gp.n_in), c->d_tables + gp.off_lo,
                          c->d_tables + gp.off_hi, gp.lo_size, sh, c->st),
           "grow kernel");
    return QUAPI_OK;
}

// The operation that adds path point n to A_in (n_in = min(n, L) digits).
quapi_status run_point(quapi_ctx* c, int64_t n, const void* A_in, void* A_out, double2* rho_slot) {
    const OpPlan* rp = nullptr;
    if (rho_slot) rp = (n <= c->L) ? &c->read_ops[n] : &c->read_steady;
    if (n < c->L) {
        if (rp) {
            quapi_status s = run_step_op(c, nullptr, rp, A_in, nullptr, rho_slot);
            if (s != QUAPI_OK) return s;
        }
        if (A_out) return run_grow_op(c, c->grow_ops[n], A_in, A_out);
        return QUAPI_OK;
    }
    const OpPlan* sp = (n == c->L) ? &c->step_first : &c->step_steady;
    if (!A_out) sp = nullptr;
    if (!sp && !rp) return QUAPI_OK;
    return run_step_op(c, sp, rp, A_in, A_out, rho_slot);
}

// Launch-shape autotuner for the steady-state step (quapi_opts.tune): times each
// candidate (TMA staging with 2, 3 or 4 stages, or plain vector loads) on the
// context's own buffers and keeps the fastest; results are cached per
// (M, L, precision, layout) for the process.
std::mutex g_tune_mutex;
std::vector<std::pair<std::string, std::pair<int, int>>> g_tune_cache;

quapi_status tune_step(quapi_ctx* c) {
    if (c->M != 2 || c->herm || c->L < 6) return QUAPI_OK;  // a single kernel shape applies there
    char keybuf[64];
    std::snprintf(keybuf, sizeof(keybuf), "M%d L%d f%d", c->M, c->L, c->form);
    const std::string key(keybuf);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (auto& kv : g_tune_cache)
            if (kv.first == key) {
                c->use_tma = kv.second.first != 0;
                c->stages = kv.second.second;
                return QUAPI_OK;
            }
    }
    const int cand[4][2] = {{1, 2}, {1, 3}, {1, 4}, {0, 2}};
    cudaEvent_t e0, e1;
    QCHECK(c, cudaEventCreate(&e0), "event");
    QCHECK(c, cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int best_i = 0;
    const int64_t n = c->L + 1;  // a steady-state step; the buffers' contents do not matter for timing
    for (int i = 0; i < 4; ++i) {
        c->use_tma = cand[i][0] != 0;
        c->stages = cand[i][1];
        quapi_status s = run_point(c, n, c->buf[0], c->buf[1], nullptr);
        if (s != QUAPI_OK) break;
        cudaEventRecord(e0, c->st);
        for (int r = 0; r < 3; ++r) {
            s = run_point(c, n, c->buf[r & 1], c->buf[(r & 1) ^ 1], nullptr);
            if (s != QUAPI_OK) break;
        }
        cudaEventRecord(e1, c->st);
        if (s != QUAPI_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->use_tma = cand[best_i][0] != 0;
    c->stages = cand[best_i][1];
    QCHECK(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st), "clear error flag");
    QCHECK(c, cudaStreamSynchronize(c->st), "tune synchronize");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.push_back({key, {cand[best_i][0], cand[best_i][1]}});
    return QUAPI_OK;
}

quapi_status check_steps(quapi_ctx* c, const int64_t* steps, int nsteps) {
    if (!steps || nsteps < 1) return fail(c, QUAPI_ERR_ARG, "steps must hold at least one entry");
    for (int i = 0; i < nsteps; ++i) {
        if (steps[i] < 0) return fail(c, QUAPI_ERR_ARG, "steps must be >= 0");
        if (i > 0 && steps[i] <= steps[i - 1]) return fail(c, QUAPI_ERR_ARG, "steps must be strictly ascending");
    }
    return QUAPI_OK;
}

// Reads (and clears) the flag a kernel sets when one of its bounded waits expired.
quapi_status check_device_error(quapi_ctx* c) {
    int flag = 0;
    QCHECK(c, cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
    if (flag) {
        QCHECK(c, cudaMemset(c->d_err, 0, sizeof(int)), "clear error flag");
        return fail(c, QUAPI_ERR_TIMEOUT, "a device-side wait gave up (copy never completed)");
    }
    return QUAPI_OK;
}

// Enqueue the whole propagation; rho(t_steps[i]) lands in slots[i] (device).
// Steps n = n_from + 1 .. N starting from A_{n_from} in buf[cur]; rho at the
// requested steps (those > n_from) lands in slots.  The newest tensor computed,
// A_{N-1}, stays in the context as its state.
quapi_status run_steps(quapi_ctx* c, int64_t n_from, int cur, const int64_t* steps, int nsteps, int next,
                       double2* slots) {
    const int64_t N = steps[nsteps - 1];
    c->state_n = n_from;
    c->state_buf = cur;
    for (int64_t n = n_from + 1; n <= N; ++n) {
        double2* slot = nullptr;
        if (next < nsteps && steps[next] == n) {
            slot = slots + (size_t)next * c->M2;
            ++next;
        }
        void* A_out = (n < N) ? c->buf[cur ^ 1] : nullptr;
        quapi_status s = run_point(c, n, c->buf[cur], A_out, slot);
        if (s != QUAPI_OK) return s;
        if (A_out) {
            cur ^= 1;
            c->state_n = n;
            c->state_buf = cur;
        }
    }
    return QUAPI_OK;
}

// Enqueue the whole propagation; rho(t_steps[i]) lands in slots[i] (device).
quapi_status propagate_enqueue(quapi_ctx* c, const double2* rho0_dev, const int64_t* steps, int nsteps,
                               double2* slots) {
    const int64_t N = steps[nsteps - 1];
    int next = 0;
    if (steps[0] == 0) {
        QCHECK(c, cudaMemcpyAsync(slots, rho0_dev, sizeof(double2) * c->M2, cudaMemcpyDeviceToDevice, c->st),
               "copy rho0");
        next = 1;
    }
    c->state_n = -1;
    if (N == 0) return QUAPI_OK;
    QCHECK(c, launch_init_tensor(rho0_dev, c->d_eta, eta_self0(c->L), c->d_s, c->M, c->form, c->buf[0], c->st,
                                 c->herm ? 1 : 0),
           "init tensor kernel");
    return run_steps(c, 0, 0, steps, nsteps, next, slots);
}

// propagate_enqueue through the context's propagation graph (see quapi_ctx::PropGraph).  A capture that
// fails (a launch that stream capture does not allow) turns the replay off for the context and runs the
// propagation directly.
quapi_status propagate_graphed(quapi_ctx* c, const double2* rho0_dev, const int64_t* steps, int nsteps,
                               double2* slots) {
    auto& g = c->graph;
    const bool same = g.rho0 == rho0_dev && g.slots == slots && g.steps.size() == (size_t)nsteps &&
                      std::equal(steps, steps + nsteps, g.steps.begin());
    if (!c->graphs || !same) {
        g.ready = false;
        g.rho0 = rho0_dev;
        g.slots = slots;
        g.steps.assign(steps, steps + nsteps);
        return propagate_enqueue(c, rho0_dev, steps, nsteps, slots);
    }
    if (!g.ready) {
        if ((!g.cap && cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess) ||
            cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graphs = false;
            return propagate_enqueue(c, rho0_dev, steps, nsteps, slots);
        }
        cudaStream_t user = c->st;
        c->st = g.cap;
        const uint64_t l0 = launches_so_far();
        const quapi_status s = propagate_enqueue(c, rho0_dev, steps, nsteps, slots);
        c->st = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g.cap, &graph);
        cudaGraphExec_t exec = nullptr;
        const bool ok = s == QUAPI_OK && e == cudaSuccess && graph &&
                        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();  // a refused capture leaves no sticky error
            uncount_launches(launches_so_far() - l0);  // recorded, never run: the direct run counts its own
            c->graphs = false;
            return propagate_enqueue(c, rho0_dev, steps, nsteps, slots);
        }
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = exec;
        g.launches = launches_so_far() - l0;
        g.state_n = c->state_n;
        g.state_buf = c->state_buf;
        g.ready = true;
        QCHECK(c, cudaGraphLaunch(g.exec, c->st), "graph launch");
        return QUAPI_OK;  // the captured launches were counted as they were recorded
    }
    QCHECK(c, cudaGraphLaunch(g.exec, c->st), "graph launch");
    count_launch(g.launches);
    c->state_n = g.state_n;
    c->state_buf = g.state_buf;
    return QUAPI_OK;
}

int64_t state_elements(const quapi_ctx* c, int64_t n) {
    const int d = (int)std::min<int64_t>(n + 1, c->L);
    return c->herm ? half_entries(c->M, d) : ipow(c->M2, d);
}

quapi_status ensure_slots(quapi_ctx* c, int nsteps) {
    if (c->slots_cap < (size_t)nsteps) {
        if (c->d_slots) cudaFree(c->d_slots);
        c->d_slots = nullptr;
        c->slots_cap = 0;
        QCHECK(c, cudaMalloc(&c->d_slots, sizeof(double2) * c->M2 * (size_t)nsteps), "cudaMalloc(rho slots)");
        c->slots_cap = nsteps;
    }
    return QUAPI_OK;
}

}  // namespace

namespace quapi {

// Launch arguments of the readout of rho(t_n) out of A_{n-1} = A_in, for entry
// points that supply their own partial-sum buffer (readout_static.cu).
quapi_status readout_launch_args(const quapi_ctx* c, int64_t n, const void* A_in, StepArgs* a, int* M,
                                 int* form, cudaStream_t* st) {
    const OpPlan* rp = (n <= c->L) ? &c->read_ops[n] : &c->read_steady;
    std::memset(a, 0, sizeof(*a));
    a->A_in = A_in;
    a->A_out = nullptr;
    a->F = ipow(c->M2, rp->n_in - 1);
    a->isum_e = c->d_tables + rp->off_isum;
    a->lo_e = c->d_tables + rp->off_lo;
    a->hi_e = c->d_tables + rp->off_hi;
    a->w_e = c->d_tables + rp->off_w;
    a->lo_size = rp->lo_size;
    int sh = 0;
    while ((int64_t(1) << sh) < rp->lo_size) ++sh;
    a->lo_shift = sh;
    a->diag_fast = rp->n_in >= 2 && rp->nk > rp->j;
    a->use_tma = c->use_tma;
    a->stages = c->stages;
    a->err_flag = c->d_err;
    a->eq_spaced = c->eq_spaced;
    a->wait_ns = c->wait_ns;
    a->fault_tx = c->fault_tx;
    a->half_digits = c->herm ? rp->n_in - 1 : -1;
    *M = c->M;
    *form = c->form;
    *st = c->st;
    return QUAPI_OK;
}

OpRef op_ref(const quapi_ctx* c, const OpPlan& p) {
    OpRef r;
    r.isum = p.summed ? c->d_tables + p.off_isum : nullptr;
    r.lo = c->d_tables + p.off_lo;
    r.hi = c->d_tables + p.off_hi;
    r.lo_size = p.lo_size;
    int sh = 0;
    while ((int64_t(1) << sh) < p.lo_size) ++sh;
    r.lo_shift = sh;
    r.hi_size = p.hi_size;
    r.n_in = p.n_in;
    r.diag = (p.n_in >= 2 && p.nk > p.j) ? 1 : 0;
    return r;
}

quapi_status batch_describe(const quapi_ctx* c, int64_t N, BatchInst* inst, int* M, int* form, cudaStream_t* st,
                            int* L) {
    std::memset(inst, 0, sizeof(*inst));
    inst->buf[0] = c->buf[0];
    inst->buf[1] = c->buf[1];
    inst->L = c->L;
    inst->N = (int)N;
    inst->herm = c->herm ? 1 : 0;
    inst->self0_idx = eta_self0(c->L);
    inst->eta = c->d_eta;
    inst->s = c->d_s;
    for (int n = 1; n < c->L; ++n) inst->grow[n] = op_ref(c, c->grow_ops[n]);
    inst->step_first = op_ref(c, c->step_first);
    inst->step = op_ref(c, c->step_steady);
    if (N >= 1) inst->read = op_ref(c, N <= c->L ? c->read_ops[N] : c->read_steady);
    *M = c->M;
    *form = c->form;
    *st = c->st;
    *L = c->L;
    return QUAPI_OK;
}

uint64_t ctx_uid(const quapi_ctx* c) { return c->uid; }
int ctx_device(const quapi_ctx* c) { return c->device; }
bool ctx_half_layout(const quapi_ctx* c) { return c->herm; }
bool ctx_tune_requested(const quapi_ctx* c) { return c->tune; }

quapi_status record_error(const quapi_ctx* c, quapi_status st, const char* msg) {
    return fail(const_cast<quapi_ctx*>(c), st, msg);
}

}  // namespace quapi

extern "C" {

void quapi_opts_init(quapi_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = QUAPI_FP64;
    o->endpoint_mode = QUAPI_ENDPOINT_STRANG;
}

quapi_status quapi_query_memory(int M, int dkmax, int precision, size_t* tensor_bytes, size_t* total_bytes) {
    if (!tensor_bytes && !total_bytes) return fail(nullptr, QUAPI_ERR_ARG, "no output pointer");
    if (M != 2 && M != 3) return fail(nullptr, QUAPI_ERR_ARG, "M must be 2 or 3");
    if (dkmax < 1 || dkmax > max_dkmax(M)) return fail(nullptr, QUAPI_ERR_ARG, "dkmax out of range");
    if (!valid_precision(precision))
        return fail(nullptr, QUAPI_ERR_ARG, "precision must be QUAPI_FP64, QUAPI_FP32 or QUAPI_DF64");
    const size_t t = 2 * (size_t)ipow(M * M, dkmax) * elem_bytes(precision);
    if (tensor_bytes) *tensor_bytes = t;
    if (total_bytes) {
        size_t tb = tables_bytes_for(M, dkmax, QUAPI_ENDPOINT_STRANG, precision);
        *total_bytes = t + tb + (size_t)16 * M * M * 152 * 16 + 4096;
    }
    return QUAPI_OK;
}

quapi_status quapi_query_memory_opts(int M, int dkmax, const quapi_opts* opts, size_t* tensor_bytes,
                                     size_t* total_bytes) {
    if (!opts) return fail(nullptr, QUAPI_ERR_ARG, "NULL opts");
    size_t t = 0, tot = 0;
    quapi_status st = quapi_query_memory(M, dkmax, opts->precision, &t, &tot);
    if (st != QUAPI_OK) return st;
    if (opts->hermitian) {
        const size_t th = 2 * (size_t)half_entries(M, dkmax) * elem_bytes(opts->precision);
        tot = tot - t + th;
        t = th;
    }
    if (!tensor_bytes && !total_bytes) return fail(nullptr, QUAPI_ERR_ARG, "no output pointer");
    if (tensor_bytes) *tensor_bytes = t;
    if (total_bytes) *total_bytes = tot;
    return QUAPI_OK;
}

quapi_status quapi_setup(const double* s, int M, const double* H, const quapi_spectral* J, double beta, double dt,
                         int dkmax, const quapi_opts* opts, quapi_ctx** out) {
    return setup_impl(s, M, H, J, beta, nullptr, dt, dkmax, opts, out);
}

quapi_status quapi_setup_eta(const double* s, int M, const double* H, const double* eta, double dt, int dkmax,
                             const quapi_opts* opts, quapi_ctx** out) {
    if (!eta) return fail(nullptr, QUAPI_ERR_ARG, "eta must not be NULL");
    for (int i = 0; i < 2 * (4 * dkmax + 3) && dkmax >= 1 && dkmax <= 16; ++i)
        if (!std::isfinite(eta[i])) return fail(nullptr, QUAPI_ERR_ARG, "eta must be finite");
    return setup_impl(s, M, H, nullptr, 1.0, eta, dt, dkmax, opts, out);
}

quapi_status quapi_propagate_device(quapi_ctx* c, const void* rho0_dev, const int64_t* steps, int nsteps,
                                    void* rho_out_dev) {
    if (!c) return fail(nullptr, QUAPI_ERR_ARG, "NULL context");
    if (!rho0_dev || !rho_out_dev) return fail(c, QUAPI_ERR_ARG, "rho0 and rho_out must not be NULL");
    if (!aligned16(rho0_dev) || !aligned16(rho_out_dev))
        return fail(c, QUAPI_ERR_ARG, "device buffers must be 16-byte aligned");
    quapi_status s = check_steps(c, steps, nsteps);
    if (s != QUAPI_OK) return s;
    return propagate_graphed(c, static_cast<const double2*>(rho0_dev), steps, nsteps,
                             static_cast<double2*>(rho_out_dev));
}

quapi_status quapi_propagate(quapi_ctx* c, const double* rho0, const int64_t* steps, int nsteps, double* rho_out) {
    if (!c) return fail(nullptr, QUAPI_ERR_ARG, "NULL context");
    if (!rho0 || !rho_out) return fail(c, QUAPI_ERR_ARG, "rho0 and rho_out must not be NULL");
    if (c->herm) {
        for (int r = 0; r < c->M; ++r)
            for (int q = 0; q < c->M; ++q) {
                const double* a = rho0 + 2 * (r * c->M + q);
                const double* b = rho0 + 2 * (q * c->M + r);
                if (std::fabs(a[0] - b[0]) > 1e-12 || std::fabs(a[1] + b[1]) > 1e-12)
                    return fail(c, QUAPI_ERR_ARG, "the Hermitian half layout needs a Hermitian rho0");
            }
    }
    quapi_status s = check_steps(c, steps, nsteps);
    if (s != QUAPI_OK) return s;
    s = ensure_slots(c, nsteps);
    if (s != QUAPI_OK) return s;
    QCHECK(c, cudaMemcpyAsync(c->d_rho0, rho0, sizeof(double2) * c->M2, cudaMemcpyHostToDevice, c->st), "copy rho0");
    s = propagate_graphed(c, c->d_rho0, steps, nsteps, c->d_slots);
    if (s != QUAPI_OK) return s;
    QCHECK(c, cudaMemcpyAsync(rho_out, c->d_slots, sizeof(double2) * c->M2 * (size_t)nsteps, cudaMemcpyDeviceToHost,
                              c->st),
           "copy rho");
    QCHECK(c, cudaStreamSynchronize(c->st), "propagate synchronize");
    return check_device_error(c);
}

quapi_status quapi_get_state(const quapi_ctx* c, int64_t* n, void* host_buf, size_t* bytes) {
    quapi_ctx* m = const_cast<quapi_ctx*>(c);
    if (!c || !n || !bytes) return fail(m, QUAPI_ERR_ARG, "NULL argument");
    if (c->state_n < 0) return fail(m, QUAPI_ERR_ARG, "no propagation state yet (propagate to a step >= 2 first)");
    const size_t need = (size_t)state_elements(c, c->state_n) * elem_bytes(c->form);
    *n = c->state_n;
    if (!host_buf) {
        *bytes = need;
        return QUAPI_OK;
    }
    if (*bytes < need) return fail(m, QUAPI_ERR_ARG, "state buffer too small");
    *bytes = need;
    QCHECK(m, cudaMemcpyAsync(host_buf, c->buf[c->state_buf], need, cudaMemcpyDeviceToHost, c->st), "copy state");
    QCHECK(m, cudaStreamSynchronize(c->st), "synchronize");
    return QUAPI_OK;
}

quapi_status quapi_set_state(quapi_ctx* c, int64_t n, const void* host_buf, size_t bytes) {
    if (!c || !host_buf) return fail(c, QUAPI_ERR_ARG, "NULL argument");
    if (n < 0) return fail(c, QUAPI_ERR_ARG, "n must be >= 0");
    const size_t need = (size_t)state_elements(c, n) * elem_bytes(c->form);
    if (bytes != need) return fail(c, QUAPI_ERR_ARG, "state size does not match (M^2)^min(n+1,L) entries");
    QCHECK(c, cudaMemcpyAsync(c->buf[0], host_buf, need, cudaMemcpyHostToDevice, c->st), "copy state");
    c->state_n = n;
    c->state_buf = 0;
    return QUAPI_OK;
}

quapi_status quapi_propagate_resume(quapi_ctx* c, const int64_t* steps, int nsteps, double* rho_out) {
    if (!c) return fail(nullptr, QUAPI_ERR_ARG, "NULL context");
    if (!rho_out) return fail(c, QUAPI_ERR_ARG, "rho_out must not be NULL");
    quapi_status s = check_steps(c, steps, nsteps);
    if (s != QUAPI_OK) return s;
    if (c->state_n < 0) return fail(c, QUAPI_ERR_ARG, "no state to resume from");
    if (steps[0] <= c->state_n) return fail(c, QUAPI_ERR_ARG, "resume steps must lie after the state's step");
    s = ensure_slots(c, nsteps);
    if (s != QUAPI_OK) return s;
    s = run_steps(c, c->state_n, c->state_buf, steps, nsteps, 0, c->d_slots);
    if (s != QUAPI_OK) return s;
    QCHECK(c, cudaMemcpyAsync(rho_out, c->d_slots, sizeof(double2) * c->M2 * (size_t)nsteps, cudaMemcpyDeviceToHost,
                              c->st),
           "copy rho");
    QCHECK(c, cudaStreamSynchronize(c->st), "resume synchronize");
    return check_device_error(c);
}

quapi_status quapi_step_device(quapi_ctx* c, int64_t n, const void* A_in_dev, void* A_out_dev, void* rho_dev) {
    if (!c) return fail(nullptr, QUAPI_ERR_ARG, "NULL context");
    if (n < 1) return fail(c, QUAPI_ERR_ARG, "n must be >= 1");
    if (!A_in_dev || (!A_out_dev && !rho_dev)) return fail(c, QUAPI_ERR_ARG, "need A_in and an output");
    if (!aligned16(A_in_dev) || !aligned16(A_out_dev) || !aligned16(rho_dev))
        return fail(c, QUAPI_ERR_ARG, "device buffers must be 16-byte aligned");
    return run_point(c, n, A_in_dev, A_out_dev, static_cast<double2*>(rho_dev));
}

quapi_status quapi_get_eta(const quapi_ctx* c, double* eta_out) {
    if (!c || !eta_out) return fail(const_cast<quapi_ctx*>(c), QUAPI_ERR_ARG, "NULL argument");
    quapi_ctx* m = const_cast<quapi_ctx*>(c);
    QCHECK(m, cudaMemcpyAsync(eta_out, c->d_eta, sizeof(double2) * (4 * c->L + 3), cudaMemcpyDeviceToHost, c->st),
           "copy eta");
    QCHECK(m, cudaStreamSynchronize(c->st), "synchronize");
    return QUAPI_OK;
}

quapi_status quapi_get_propagator(const quapi_ctx* c, double* U_out, double* K_out) {
    if (!c || !U_out) return fail(const_cast<quapi_ctx*>(c), QUAPI_ERR_ARG, "NULL argument");
    quapi_ctx* m = const_cast<quapi_ctx*>(c);
    QCHECK(m, cudaMemcpyAsync(U_out, c->d_U, sizeof(double2) * c->M * c->M, cudaMemcpyDeviceToHost, c->st), "copy U");
    if (K_out)
        QCHECK(m, cudaMemcpyAsync(K_out, c->d_K, sizeof(double2) * c->M2 * c->M2, cudaMemcpyDeviceToHost, c->st),
               "copy K");
    QCHECK(m, cudaStreamSynchronize(c->st), "synchronize");
    return QUAPI_OK;
}

uint64_t quapi_kernel_launches(void) { return launches_so_far(); }

const char* quapi_last_error(const quapi_ctx* c) {
    if (c) return c->err.c_str();
    return g_thread_error.c_str();
}

void quapi_destroy(quapi_ctx* c) {
    if (!c) return;
    batch_forget(c->uid);
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    cudaFree(c->d_s);
    cudaFree(c->d_H);
    cudaFree(c->d_U);
    cudaFree(c->d_K);
    cudaFree(c->d_eta);
    cudaFree(c->d_rho0);
    cudaFree(c->d_slots);
    if (c->own_buf) {
        cudaFree(c->buf[0]);
        cudaFree(c->buf[1]);
    }
    cudaFree(c->d_tables);
    cudaFree(c->d_partial);
    cudaFree(c->d_err);
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    if (c->graph.cap) cudaStreamDestroy(c->graph.cap);
    delete c;
}

}  // extern "C"
