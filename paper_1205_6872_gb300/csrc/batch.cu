// Batched propagation: many independent instances (own L, eta, K, N) in one
// persistent kernel launch, captured once into a CUDA graph and replayed.
//
// Work list.  Instances whose two tensors fit in 32 KB of shared memory
// ("resident") run in a kernel of their own, one CTA per instance doing all of
// its steps in shared memory, on a side branch of the graph (concurrent with the
// tiled kernel, which then carries neither their code nor their shared memory).
// Every other instance contributes, for each step n, ceil(tiles / group) items
// of `group` tiles (a tile = 256 x FPT fibers or growth entries).  Items are
// numbered step-major (wave n = step n of every instance), so an item only ever
// depends on items with smaller numbers: a CTA takes the next number from an atomic counter,
// looks up its (step, instance, first tile) in a flat item table, waits
// (bounded) until its instance has completed every tile of the previous step,
// takes the number of its following item (the atomic's latency then overlaps
// the tiles), processes its tiles, and publishes the count.  The readout at the
// instance's final step writes one partial sum per tile; the CTA finishing the
// last tile adds them in tile order (deterministic result).
//
// Dynamic shared memory is sized to the largest resident instance (none: 0), and a batch whose tiled
// instances all use the Hermitian half layout runs a kernel without the full-layout tile code.
//
// Launch shape (FPT, group) is chosen per batch signature by timing candidates
// when tuning is requested (quapi_opts.tune or QUAPI_TUNE=1); the choice is
// cached in memory and, if QUAPI_TUNE_CACHE names a file, on disk.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "batch_kernel.cuh"

namespace quapi {

namespace {

using namespace batchk;

// ------------------------------------------------------------------ host side

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

struct Plan {
    int M = 0, form = 0, fpt = 0, group = 0, n = 0;
    std::vector<uint64_t> uids;
    std::vector<int64_t> Ns;
    std::vector<BatchInst> inst;
    std::vector<int> resident, tiled;
    int nwaves = 0;
    int64_t total_items = 0;
    DevBuf d_inst, d_res, d_tiled, d_wave, d_items, d_need, d_nt, d_next, d_err, d_cnt, d_part, d_rho0, d_rho;
    double* h_rho0 = nullptr;  // pinned staging
    double* h_rho = nullptr;
    BatchLaunch launch;        // kernel arguments, launch shape and layout flag
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t cnt_bytes = 0;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        if (launch.side) cudaStreamDestroy(launch.side);
        if (launch.fork) cudaEventDestroy(launch.fork);
        if (launch.join) cudaEventDestroy(launch.join);
        if (h_rho0) cudaFreeHost(h_rho0);
        if (h_rho) cudaFreeHost(h_rho);
    }
};

std::mutex g_plans_mutex;
std::map<std::string, Plan*> g_plans;
std::map<std::string, std::pair<int, int>> g_tuned;  // signature -> (fpt, group)

std::string plan_key(const std::vector<uint64_t>& uids, const std::vector<int64_t>& Ns, int fpt, int group) {
    std::ostringstream o;
    o << fpt << ":" << group;
    for (size_t i = 0; i < uids.size(); ++i) o << "|" << uids[i] << "," << Ns[i];
    return o.str();
}

int64_t ipow64(int64_t b, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// canonical prefixes of n digits in the half layout: ((M^2)^n + M^n) / 2
int64_t canon64(int M, int n) { return (ipow64((int64_t)M * M, n) + ipow64(M, n)) >> 1; }

// tiles of instance (L, N) at step n for the given tile size
unsigned tiles_at(int M2, int L, int64_t N, int n, int te, int read_nin, bool herm) {
    if (n < 1 || n > N) return 0;
    int64_t units;
    if (herm) {
        const int M = M2 == 4 ? 2 : 3;
        if (n < L && n < N) units = M2 * canon64(M, n - 1);     // growth: stored input entries
        else if (n < N) units = canon64(M, L - 1);              // step: canonical prefixes
        else units = canon64(M, read_nin - 1);                  // readout: canonical prefixes
    } else {
        if (n < L && n < N) units = ipow64(M2, n);              // growth: input entries
        else if (n < N) units = ipow64(M2, L - 1);              // step: fibers
        else units = ipow64(M2, read_nin - 1);                  // readout: fibers
    }
    return (unsigned)((units + te - 1) / te);
}

// kernels one run launches: the resident instances' kernel, the tiled instances' init and main kernels
uint64_t kernels_per_run(const Plan& P) {
    return (P.launch.args.nresident ? 1 : 0) + (P.launch.args.ntiled ? 2 : 0);
}

// prep = true: only set the kernel's shared-memory attribute and size the grid
cudaError_t launch_plan(Plan& P, cudaStream_t st, bool prep = false) {
    if (P.form == QUAPI_FP32) return launch_batch_fp32(P.launch, st, prep);
    if (P.form == QUAPI_FP64) return launch_batch_fp64(P.launch, st, prep);
    if (P.form == QUAPI_DF64) return launch_batch_df64(P.launch, st, prep);
    return cudaErrorInvalidValue;
}

template <class T> cudaError_t upload(DevBuf& b, const std::vector<T>& v) {
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(&b.p, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Enqueue one run of the plan: counters cleared, rho0 uploaded, kernels, rho downloaded.
cudaError_t enqueue_run(Plan& P, cudaStream_t st) {
    cudaError_t e;
    const int M2 = P.M * P.M;
    if ((e = cudaMemsetAsync(P.d_cnt.p, 0, P.cnt_bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(P.d_next.p, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(P.d_rho0.p, P.h_rho0, sizeof(double2) * M2 * P.n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_plan(P, st)) != cudaSuccess) return e;
    return cudaMemcpyAsync(P.h_rho, P.d_rho.p, sizeof(double2) * M2 * P.n, cudaMemcpyDeviceToHost, st);
}

cudaError_t build_plan(Plan& P, const std::vector<BatchInst>& insts, int M, int form, int fpt, int group,
                       uint64_t wait_ns) {
    cudaError_t e;
    const int M2 = M * M;
    const size_t elt = form == QUAPI_FP32 ? 8 : 16;  // complex float; complex double or double-float pair
    if (fpt == 8 && !(M == 2 && form == QUAPI_FP32)) fpt = 4;  // 8 fibers per thread: M = 2 FP32 only
    P.M = M;
    P.form = form;
    P.fpt = fpt;
    P.group = group;
    P.n = (int)insts.size();
    P.inst = insts;
    P.launch.M = M;
    P.launch.fpt = fpt;
    P.launch.smem = 0;  // the largest resident instance's two tensors (none: no dynamic shared memory)
    const int te = kBThreads * fpt;
    // the resident instances' kernel runs on a side stream, forked from and joined to the main one
    if ((e = cudaStreamCreateWithFlags(&P.launch.side, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&P.launch.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&P.launch.join, cudaEventDisableTiming)) != cudaSuccess) return e;
    // per-instance buffers
    if ((e = cudaMalloc(&P.d_rho0.p, sizeof(double2) * M2 * P.n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.d_rho.p, sizeof(double2) * M2 * P.n)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&P.h_rho0, sizeof(double2) * M2 * P.n)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&P.h_rho, sizeof(double2) * M2 * P.n)) != cudaSuccess) return e;
    std::vector<int64_t> read_tiles(P.n, 0);
    int64_t part_total = 0;
    for (int i = 0; i < P.n; ++i) {
        BatchInst& I = P.inst[i];
        const bool res = 2 * (size_t)ipow64(M2, I.L) * elt <= (size_t)kResidentBytes;
        if (res) {
            P.resident.push_back(i);
            P.launch.smem = std::max(P.launch.smem, 2 * (size_t)ipow64(M2, I.L) * elt);
        } else {
            P.tiled.push_back(i);
            read_tiles[i] = tiles_at(M2, I.L, I.N, I.N, te, I.read.n_in, I.herm != 0);
            part_total += read_tiles[i];
        }
    }
    P.launch.half_only = M == 2 && !P.tiled.empty();
    for (int i : P.tiled) P.launch.half_only = P.launch.half_only && P.inst[i].herm != 0;
    // counters (done + read_done per instance) and readout partials
    P.cnt_bytes = sizeof(unsigned) * 2 * std::max(P.n, 1);
    if ((e = cudaMalloc(&P.d_cnt.p, P.cnt_bytes)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.d_part.p, sizeof(double2) * M2 * std::max<int64_t>(part_total, 1))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&P.d_next.p, sizeof(unsigned long long))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&P.d_err.p, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(P.d_err.p, 0, sizeof(int))) != cudaSuccess) return e;
    unsigned* cnt = static_cast<unsigned*>(P.d_cnt.p);
    double2* part = static_cast<double2*>(P.d_part.p);
    int64_t poff = 0;
    for (int i = 0; i < P.n; ++i) {
        BatchInst& I = P.inst[i];
        I.done = cnt + 2 * i;
        I.read_done = cnt + 2 * i + 1;
        I.rho0 = static_cast<double2*>(P.d_rho0.p) + (size_t)M2 * i;
        I.rho_out = static_cast<double2*>(P.d_rho.p) + (size_t)M2 * i;
        I.partial = part + poff * M2;
        poff += read_tiles[i];
    }
    // work list
    int nw = 0;
    for (int i : P.tiled) nw = std::max<int>(nw, P.inst[i].N);
    P.nwaves = nw;
    const int nt = (int)P.tiled.size();
    std::vector<int64_t> wave_off(nw + 2, 0);
    std::vector<uint4> items;  // tiled items in work-list order
    std::vector<unsigned> need((size_t)(nw + 1) * std::max(nt, 1), 0), ntl((size_t)(nw + 1) * std::max(nt, 1), 0);
    wave_off[0] = 0;
    wave_off[1] = 0;  // resident instances run in their own kernel; the tiled items are numbered from 0
    std::vector<unsigned> cum(nt, 0);
    for (int n = 1; n <= nw; ++n) {
        int64_t acc = 0;
        for (int k = 0; k < nt; ++k) {
            const BatchInst& I = P.inst[P.tiled[k]];
            const unsigned t = tiles_at(M2, I.L, I.N, n, te, I.read.n_in, I.herm != 0);
            ntl[(size_t)n * nt + k] = t;
            need[(size_t)n * nt + k] = cum[k];
            for (unsigned t0 = 0; t0 < t; t0 += (unsigned)group) items.push_back(make_uint4((unsigned)n, (unsigned)k, t0, 0u));
            acc += (t + group - 1) / group;
            cum[k] += t;
        }
        wave_off[n + 1] = wave_off[n] + acc;
    }
    P.total_items = wave_off[nw + 1];
    if (nw == 0) P.total_items = wave_off[1];
    if (const char* f = std::getenv("QUAPI_FAULT")) {
        // host-side fault injection: the first tiled instance's step 2 waits for a count nothing reaches
        if (std::strcmp(f, "batch_wait") == 0 && nt > 0 && nw >= 2) need[(size_t)2 * nt + 0] = 0xFFFFFFFFu;
    }
    if ((e = upload(P.d_inst, P.inst)) != cudaSuccess) return e;
    if ((e = upload(P.d_res, P.resident)) != cudaSuccess) return e;
    if ((e = upload(P.d_tiled, P.tiled)) != cudaSuccess) return e;
    if ((e = upload(P.d_wave, wave_off)) != cudaSuccess) return e;
    if ((e = upload(P.d_items, items)) != cudaSuccess) return e;
    if ((e = upload(P.d_need, need)) != cudaSuccess) return e;
    if ((e = upload(P.d_nt, ntl)) != cudaSuccess) return e;
    BatchArgs& a = P.launch.args;
    a.inst = static_cast<const BatchInst*>(P.d_inst.p);
    a.resident = static_cast<const int*>(P.d_res.p);
    a.nresident = (int)P.resident.size();
    a.tiled = static_cast<const int*>(P.d_tiled.p);
    a.ntiled = nt;
    a.nwaves = nw;
    a.wave_off = static_cast<const int64_t*>(P.d_wave.p);
    a.items = static_cast<const uint4*>(P.d_items.p);
    a.need = static_cast<const unsigned*>(P.d_need.p);
    a.ntiles = static_cast<const unsigned*>(P.d_nt.p);
    a.total_items = P.total_items;
    a.next_item = static_cast<unsigned long long*>(P.d_next.p);
    a.err = static_cast<int*>(P.d_err.p);
    a.group = group;
    a.wait_ns = wait_ns;
    return cudaSuccess;
}

// (M, form, and the sorted (L, N, layout) of the instances): batches with the same signature share a
// tuned launch shape
std::string signature(const std::vector<BatchInst>& insts, int M, int form) {
    std::vector<std::tuple<int, int64_t, int>> v;
    for (const auto& I : insts) v.emplace_back(I.L, (int64_t)I.N, I.herm);
    std::sort(v.begin(), v.end());
    std::ostringstream o;
    o << "M" << M << "f" << form;
    for (auto& p : v) o << ";" << std::get<0>(p) << "," << std::get<1>(p) << (std::get<2>(p) ? "h" : "");
    return o.str();
}

bool tune_cache_lookup(const std::string& sig, int& fpt, int& group) {
    auto it = g_tuned.find(sig);
    if (it != g_tuned.end()) {
        fpt = it->second.first;
        group = it->second.second;
        return true;
    }
    const char* path = std::getenv("QUAPI_TUNE_CACHE");
    if (!path) return false;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string s;
        int f, g;
        if (ls >> s >> f >> g && s == sig) {
            fpt = f;
            group = g;
            g_tuned[sig] = {f, g};
            return true;
        }
    }
    return false;
}

void tune_cache_store(const std::string& sig, int fpt, int group) {
    g_tuned[sig] = {fpt, group};
    if (const char* path = std::getenv("QUAPI_TUNE_CACHE")) {
        std::ofstream out(path, std::ios::app);
        out << sig << " " << fpt << " " << group << "\n";
    }
}

uint64_t wait_limit_ns() {
    if (const char* v = std::getenv("QUAPI_WAIT_MS")) {
        const double ms = std::atof(v);
        if (ms > 0) return (uint64_t)(ms * 1e6);
    }
    return 2000000000ull;
}

}  // namespace

// Frees every cached batch plan that includes the context with this uid.
void batch_forget(uint64_t uid) {
    std::lock_guard<std::mutex> lock(g_plans_mutex);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        Plan* P = it->second;
        if (std::find(P->uids.begin(), P->uids.end(), uid) != P->uids.end()) {
            delete P;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace quapi

using namespace quapi;

extern "C" quapi_status quapi_propagate_batch(int n, quapi_ctx* const* ctxs, const double* const* rho0s,
                                              const int64_t* nsteps_each, double* const* rho_final) {
    if (n < 1 || !ctxs || !rho0s || !nsteps_each || !rho_final)
        return record_error(nullptr, QUAPI_ERR_ARG, "batch: n >= 1 and non-NULL arrays required");
    std::vector<BatchInst> insts(n);
    std::vector<uint64_t> uids(n);
    std::vector<int64_t> Ns(n);
    int M0 = 0, form0 = 0, L = 0;
    cudaStream_t st0 = nullptr;
    bool tune = false;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !rho0s[i] || !rho_final[i])
            return record_error(nullptr, QUAPI_ERR_ARG, "batch: NULL context or buffer");
        if (nsteps_each[i] < 0) return record_error(nullptr, QUAPI_ERR_ARG, "batch: final steps must be >= 0");
        int M, form;
        cudaStream_t st;
        batch_describe(ctxs[i], nsteps_each[i], &insts[i], &M, &form, &st, &L);
        if (i == 0) {
            M0 = M;
            form0 = form;
            st0 = st;
        } else if (M != M0 || form != form0) {
            return record_error(nullptr, QUAPI_ERR_UNSUPPORTED, "batch: all contexts need the same M and precision");
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return record_error(nullptr, QUAPI_ERR_ARG, "batch: a context appears twice");
        if (ctx_half_layout(ctxs[i])) {  // the half layout stores one of each conjugate pair: rho0 = rho0^dagger
            const double* r0 = rho0s[i];
            for (int r = 0; r < M; ++r)
                for (int q = 0; q < M; ++q) {
                    const double* a = r0 + 2 * (r * M + q);
                    const double* b = r0 + 2 * (q * M + r);
                    if (std::fabs(a[0] - b[0]) > 1e-12 || std::fabs(a[1] + b[1]) > 1e-12)
                        return record_error(nullptr, QUAPI_ERR_ARG, "batch: the Hermitian half layout needs a Hermitian rho0");
                }
        }
        uids[i] = ctx_uid(ctxs[i]);
        Ns[i] = nsteps_each[i];
    }
    if (const char* v = std::getenv("QUAPI_TUNE")) tune = std::atoi(v) != 0;
    tune = tune || ctx_tune_requested(ctxs[0]);
    const int M2 = M0 * M0;
    // instances that stop at step 0 return rho0 unchanged and stay out of the kernel
    std::vector<int> active;
    for (int i = 0; i < n; ++i) {
        if (Ns[i] == 0) std::memcpy(rho_final[i], rho0s[i], sizeof(double) * 2 * M2);
        else active.push_back(i);
    }
    if (active.empty()) return QUAPI_OK;
    std::vector<BatchInst> act;
    std::vector<uint64_t> auids;
    std::vector<int64_t> aNs;
    for (int i : active) {
        act.push_back(insts[i]);
        auids.push_back(uids[i]);
        aNs.push_back(Ns[i]);
    }
    const std::string sig = signature(act, M0, form0);
    const uint64_t wait_ns = wait_limit_ns();

    std::lock_guard<std::mutex> lock(g_plans_mutex);
    int fpt = form0 == QUAPI_FP32 ? 2 : 1, group = 4;
    auto get_plan = [&](int f, int g, Plan** out) -> cudaError_t {
        const std::string key = plan_key(auids, aNs, f, g);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            *out = it->second;
            return cudaSuccess;
        }
        Plan* P = new Plan();
        P->uids = auids;
        P->Ns = aNs;
        cudaError_t e = build_plan(*P, act, M0, form0, f, g, wait_ns);
        if (e != cudaSuccess) {
            delete P;
            return e;
        }
        g_plans[key] = P;
        *out = P;
        return cudaSuccess;
    };
    if (tune && !tune_cache_lookup(sig, fpt, group)) {
        // time every candidate launch shape once (after a warm-up run) and keep the fastest
        const int fpts[4] = {1, 2, 4, 8};  // 8: M = 2 FP32 only (other batches run it as 4)
        const int groups[4] = {1, 4, 8, 16};
        float best = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int f : fpts)
            for (int g : groups) {
                if (f == 8 && !(M0 == 2 && form0 == QUAPI_FP32)) continue;
                Plan* P = nullptr;
                if (get_plan(f, g, &P) != cudaSuccess) continue;
                for (size_t j = 0; j < active.size(); ++j)
                    std::memcpy(P->h_rho0 + 2 * M2 * j, rho0s[active[j]], sizeof(double) * 2 * M2);
                if (enqueue_run(*P, st0) != cudaSuccess) continue;
                cudaEventRecord(e0, st0);
                if (enqueue_run(*P, st0) != cudaSuccess) continue;
                cudaEventRecord(e1, st0);
                count_launch(2 * kernels_per_run(*P));
                if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    fpt = f;
                    group = g;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune_cache_store(sig, fpt, group);
    }
    Plan* P = nullptr;
    cudaError_t e = get_plan(fpt, group, &P);
    if (e != cudaSuccess)
        return record_error(nullptr, e == cudaErrorMemoryAllocation ? QUAPI_ERR_OOM : QUAPI_ERR_CUDA,
                            cudaGetErrorString(e));
    for (size_t j = 0; j < active.size(); ++j)
        std::memcpy(P->h_rho0 + 2 * M2 * j, rho0s[active[j]], sizeof(double) * 2 * M2);
    if (!P->exec) {
        // capture the whole run (counter resets, copies, both kernels) once; replay it afterwards
        if ((e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking)) != cudaSuccess)
            return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
        if ((e = launch_plan(*P, P->cap, true)) != cudaSuccess)  // attributes and grid, outside the capture
            return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
        cudaError_t ee = enqueue_run(*P, P->cap);
        e = cudaStreamEndCapture(P->cap, &graph);
        if (ee != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(ee != cudaSuccess ? ee : e));
        }
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    }
    if ((e = cudaGraphLaunch(P->exec, st0)) != cudaSuccess)
        return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    count_launch(kernels_per_run(*P));
    if ((e = cudaStreamSynchronize(st0)) != cudaSuccess)
        return record_error(nullptr, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    int flag = 0;
    cudaMemcpy(&flag, P->d_err.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) {
        cudaMemset(P->d_err.p, 0, sizeof(int));
        return record_error(nullptr, QUAPI_ERR_TIMEOUT, "batch: a dependency wait gave up");
    }
    for (size_t j = 0; j < active.size(); ++j)
        std::memcpy(rho_final[active[j]], P->h_rho + 2 * M2 * j, sizeof(double) * 2 * M2);
    return QUAPI_OK;
}
