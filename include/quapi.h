/* quapi.h -- C ABI of the GB300-native QUAPI tensor-propagator library (libquapi.so).
 *
 * The library evaluates the reduced density matrix of an open quantum system in
 * the Feynman-Vernon model (Sec. II: H = H_OQS + sum_k c_k s Q_k + bath of
 * harmonic oscillators, spectral density J(w), Eq. spectralDistribution) by the
 * quasi-adiabatic propagator path integral in tensor-propagator form (Sec. I):
 * the discretised path sum of Sec. II with memory truncated at Delta k_max
 * ("dkmax", written L below), time step dt, and the eta coefficients of
 * Eqs. etaKK'generalTrotter .. etaNkgeneralStrang.  The user supplies what
 * Sec. II lists as the program's inputs: the coordinate vector s, H_OQS, J(w)
 * and the temperature, rho(0), a grid of times t_k = k dt, and {dt, L}
 * (hbar = k_B = 1; the temperature is passed as beta = 1/T).
 *
 * Conventions used by every entry point
 *   - Complex numbers are interleaved (re, im) doubles on the host.
 *   - A path point x = (s^+, s^-) of an M-level system is the flat index
 *     x = i_plus * M + i_minus, i.e. rho is an M x M row-major matrix.
 *   - The augmented tensor A (device) has (M^2)^L complex entries; digit p of
 *     its flat index (base M^2, p = 0 least significant) holds the path point
 *     k - L + 1 + p, so the oldest point is contiguous.  FP64 form: complex
 *     double (16 B); FP32 form: complex float (8 B); DF64 form: four floats
 *     {re_hi, im_hi, re_lo, im_lo} (16 B) with value (re_hi + re_lo) + i (im_hi + im_lo).
 *   - The caller owns every host array it passes; the library copies what it
 *     needs and keeps no caller pointer beyond the call.  Device memory that
 *     the library allocates is owned by the context and released by
 *     quapi_destroy.  A caller-supplied workspace stays caller-owned.
 *   - Every function returns a quapi_status; nothing aborts or exits.  On
 *     error, quapi_last_error(ctx) (or quapi_last_error(NULL) for errors
 *     raised before a context exists) describes it.
 *   - One context is used by one host thread at a time.
 */
#ifndef QUAPI_H
#define QUAPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct quapi_ctx quapi_ctx;

typedef enum {
    QUAPI_OK = 0,
    QUAPI_ERR_ARG = 1,          /* invalid argument (non-Hermitian H, M not 2 or 3, dt <= 0, ...) */
    QUAPI_ERR_OOM = 2,          /* device memory (or the caller's workspace) too small */
    QUAPI_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed */
    QUAPI_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up (batched kernel, TMA-staged step) */
    QUAPI_ERR_UNSUPPORTED = 5   /* valid request this build does not implement */
} quapi_status;

/* Spectral densities J(w) (Eq. spectralDistribution): two parametric forms, or a table. */
typedef enum {
    QUAPI_J_OHMIC_EXP = 0,        /* J = (pi/2) a w exp(-w/wc)                               */
    QUAPI_J_SUPEROHMIC_GAUSS = 1, /* J = a w^3 exp(-(w/wc)^2)  (Eq. superOhmicJwithGaussianCutoff) */
    QUAPI_J_TABULATED = 2         /* J given at n frequencies: piecewise linear through (0, 0) and
                                     (omega[i], values[i]), zero above omega[n-1]               */
} quapi_jkind;

typedef struct {
    int kind;    /* quapi_jkind */
    double a;    /* parametric kinds: prefactor (alpha for Ohmic, xi / A for super-Ohmic), >= 0 */
    double wc;   /* parametric kinds: cutoff frequency, > 0 */
    /* QUAPI_J_TABULATED only (ignored otherwise).  Host arrays owned by the caller and read
       during quapi_setup only.  omega: n strictly ascending finite frequencies, omega[0] > 0;
       values: J at those frequencies, finite and >= 0; 1 <= n <= 65536.  The eta integrals run
       over [0, omega[n-1]] with quadrature panels aligned to the table's nodes.  Any violation
       is QUAPI_ERR_ARG. */
    const double* omega;
    const double* values;
    int n;
} quapi_spectral;

enum {
    QUAPI_FP64 = 64,  /* tensor stored and propagated in complex double */
    QUAPI_FP32 = 32,  /* complex float storage and products; double-float tables,
                         compensated index sums (FP32 products of the tables' hi
                         floats inside the sums once K sits in the hi table; the
                         factors that carry K keep both floats), FP64 eta / K /
                         readout */
    QUAPI_DF64 = 48   /* FP64-equivalent form on the FP32 pipes: each entry stored as a
                         double-float pair (hi + lo floats, 16 B per complex entry, ~48-bit
                         significands), triple-float tables holding the FP64 values exactly,
                         error-free products and sums; FP64 readout */
};

enum {
    QUAPI_ENDPOINT_STRANG = 0,   /* rho(t_N) with the half end box of Eqs. etaNNgeneralStrang,
                                    etaNkgeneralStrang, etaN0generalStrang (default)            */
    QUAPI_ENDPOINT_INTERIOR = 1  /* rho(t_N) with the final point treated as an interior point  */
};

typedef struct {
    int precision;          /* QUAPI_FP64 (default), QUAPI_FP32 or QUAPI_DF64                      */
    int endpoint_mode;      /* QUAPI_ENDPOINT_STRANG (default) or QUAPI_ENDPOINT_INTERIOR           */
    void* cuda_stream;      /* cudaStream_t all work is issued on; NULL = the legacy default stream */
    int tune;               /* 0: default launch shape; 1: pick it by timing candidates (cached)   */
    void* workspace;        /* optional caller-owned device buffer for the tensors (16-byte
                               aligned), or NULL                                                  */
    size_t workspace_bytes; /* its size; must be >= quapi_query_memory_opts()'s tensor_bytes       */
    int hermitian;          /* 1: keep only (about) half of A (M = 2 or 3; needs a Hermitian rho0).
                               Swapping s+ and s- at every path point conjugates a path's weight, so
                               A(conj path) = conj(A(path)): point x = (a, b) = a*M + b goes to
                               (b, a).  Points with a = b are self-conjugate; of each other pair the
                               point with a < b is canonical (M = 2: 0=(+,+) 1=(+,-) 2=(-,+) 3=(-,-),
                               canonical 1, self-conjugate 0 and 3; M = 3: canonical 1, 2, 5 with
                               conjugates 3, 6, 7, self-conjugate 0, 4, 8).  A prefix is canonical
                               when its first digit that is not self-conjugate is canonical;
                               canonical prefixes of n digits are ordered [each canonical top point in
                               increasing order: (M^2)^(n-1) plain continuations][each self-
                               conjugate top point in increasing order: canonical n-1].  An n-digit
                               tensor stores the M^2-entry last-digit fiber of every canonical
                               (n-1)-digit prefix, in that order: M^2 ((M^2)^(n-1) + M^(n-1))/2
                               entries (M = 2: 2*4^(n-1) + 2^n), prefix c at entry M^2 c.  Tensors
                               passed to quapi_step_device / quapi_readout_static and the checkpoint
                               state use this layout; quapi_propagate_batch keeps it for the
                               instance's tensors. */
} quapi_opts;

/* Fill *opts with the defaults above. */
void quapi_opts_init(quapi_opts* opts);

/* Device memory a context needs (Sec. II, Eq. memoryComplexity: the stored
 * tensors grow as M^{2 L}).  tensor_bytes: the two ping-pong copies of A
 * (2 (M^2)^L elements), which a caller workspace must hold; total_bytes adds
 * the tables and readout scratch the library allocates itself.
 * Errors: QUAPI_ERR_ARG for M not in {2,3}, L < 1, L beyond the index range,
 * unknown precision, or a NULL output pointer. */
quapi_status quapi_query_memory(int M, int dkmax, int precision, size_t* tensor_bytes,
                                size_t* total_bytes);

/* As quapi_query_memory, for the precision and layout in *opts (opts->precision, opts->hermitian;
 * the other fields are ignored): with the Hermitian half layout tensor_bytes is the two copies of
 * its M^2 ((M^2)^(L-1) + M^(L-1))/2 stored entries, the size a caller workspace needs for it.
 * Errors: as quapi_query_memory; QUAPI_ERR_ARG for a NULL opts. */
quapi_status quapi_query_memory_opts(int M, int dkmax, const quapi_opts* opts, size_t* tensor_bytes,
                                     size_t* total_bytes);

/* Set up one problem (Sec. II's inputs).
 *   s      [M]        coordinate eigenvalues (real), the basis H is given in
 *   M      2 or 3
 *   H      [M*M]      complex, row-major, Hermitian to 1e-12 (absolute)
 *   J      spectral density parameters; beta > 0 (1/T); dt > 0; dkmax = L >= 1
 *   opts   NULL for defaults
 * On the device (FP64): U = exp(-i H dt) and the pair propagator
 * K(x', x) = U[a',a] conj(U[b',b]) (the bare propagators of the path-integral
 * expression, Sec. II); the 4L+3 eta coefficients by Gauss-Legendre
 * quadrature of their frequency-integral form (Eq. bathResponseFunction,
 * Eqs. etaKK'generalTrotter .. etaNkgeneralStrang, symmetric box placement);
 * the influence-functional factor tables (Sec. II, Eq. for I).
 * Returns a context in *out (NULL on error).
 * Errors: QUAPI_ERR_ARG (bad sizes, non-Hermitian H, dt/beta <= 0, unknown J
 * kind), QUAPI_ERR_OOM, QUAPI_ERR_CUDA. */
quapi_status quapi_setup(const double* s, int M, const double* H, const quapi_spectral* J,
                         double beta, double dt, int dkmax, const quapi_opts* opts,
                         quapi_ctx** out);

/* As quapi_setup, but with the eta coefficients supplied by the caller (the
 * paper's alternative of giving alpha(t) instead of J(w), Sec. II).
 *   eta [4L+3] complex, in this order:
 *     interior[dk], dk = 0..L   eta between two interior points dk apart (dk = 0: self term)
 *     point0[k-1],  k = 1..L    eta_{k0} (Eq. etaK0generalStrang)
 *     end_self                  eta_NN   (Eq. etaNNgeneralStrang)
 *     end[dk-1],    dk = 1..L   eta_{N,N-dk} (Eq. etaNkgeneralStrang)
 *     end_point0[N-1], N = 1..L eta_{N0}  (Eq. etaN0generalStrang)
 *     self0                     eta_00    (Eq. eta00generalStrang)
 * Errors as quapi_setup. */
quapi_status quapi_setup_eta(const double* s, int M, const double* H, const double* eta,
                             double dt, int dkmax, const quapi_opts* opts, quapi_ctx** out);

/* Propagate rho(0) and return rho(t_k) at the requested steps (Sec. II: "all
 * (or some)" of the times t_k = k dt; Sec. IV's allPoints / justFinalPoint).
 *   rho0     [M*M] complex (host)
 *   steps    [nsteps] step indices k >= 0, strictly ascending (host)
 *   rho_out  [nsteps*M*M] complex (host, caller-owned), rho(t_{steps[i]}) at i*M*M
 * Runs the growth phase (k < L), then the fused steady-state step, with the
 * rho readout fused into the step kernel only at the requested steps.  Blocks
 * until rho_out is written.
 * Errors: QUAPI_ERR_ARG (NULL pointers, nsteps < 1, unsorted or negative
 * steps), QUAPI_ERR_CUDA. */
quapi_status quapi_propagate(quapi_ctx* c, const double* rho0, const int64_t* steps, int nsteps,
                             double* rho_out);

/* As quapi_propagate with rho0 and rho_out in device memory (complex double,
 * 16-byte aligned), enqueued on the context's stream without a host
 * synchronisation.  steps is a host array.  Errors as quapi_propagate, and
 * QUAPI_ERR_ARG for a device pointer that is not 16-byte aligned.
 *
 * Both propagate calls replay a CUDA graph when called again with the same
 * arguments: the second call with a given (rho0 buffer, rho_out buffer, step
 * list) -- for quapi_propagate, the context's own device copies -- captures the
 * whole propagation on a private stream and launches it into the context's
 * stream; later calls with the same arguments launch that graph, which reads
 * the buffers' current contents.  Results are bitwise those of direct
 * launches.  The environment variable QUAPI_GRAPH=0, read at set-up, turns the
 * replay off for the context. */
quapi_status quapi_propagate_device(quapi_ctx* c, const void* rho0_dev, const int64_t* steps,
                                    int nsteps, void* rho_out_dev);

/* Checkpoint and resume.  After quapi_propagate(_device) to a final step N
 * the context keeps its newest tensor A_{N-1}, which holds everything the
 * recurrence needs to continue (Sec. I: the tensor propagator is Markovian in
 * the augmented tensor); quapi_propagate_resume continues from it.
 *   quapi_get_state: *n = the path point of the kept tensor; with host_buf
 *     NULL only *bytes is set to its size ((M^2)^min(n+1,L) entries in the
 *     context's storage format); otherwise *bytes (in: capacity) >= that size
 *     and the tensor is copied to host_buf (synchronous).
 *   quapi_set_state: load A_n from host_buf (bytes must equal that size) into
 *     a context set up with the same inputs; it becomes the kept tensor.
 *   quapi_propagate_resume: rho at the requested steps, all > n (ascending),
 *     continuing from the kept tensor; blocks until rho_out is written.
 * Errors: QUAPI_ERR_ARG (no state yet, size mismatch, steps not after n),
 * QUAPI_ERR_CUDA. */
quapi_status quapi_get_state(const quapi_ctx* c, int64_t* n, void* host_buf, size_t* bytes);
quapi_status quapi_set_state(quapi_ctx* c, int64_t n, const void* host_buf, size_t bytes);
quapi_status quapi_propagate_resume(quapi_ctx* c, const int64_t* steps, int nsteps, double* rho_out);

/* One tensor-propagator step on caller device buffers: the step that adds
 * path point n (n >= 1) to A_{n-1} (Sec. I, multiply by the propagator tensor
 * T and, once A_{n-1} holds L points, sum over the oldest index).
 *   A_in_dev   A_{n-1}: (M^2)^min(n,L) elements in the context's precision
 *   A_out_dev  A_n: (M^2)^min(n+1,L) elements, or NULL to skip writing it
 *   rho_dev    if not NULL, M*M complex double receiving rho(t_n) read out of
 *              A_{n-1} with the context's end-point treatment
 * Asynchronous on the context's stream.  A_in and A_out must not overlap.
 * Every device pointer must be 16-byte aligned (cudaMalloc and PyTorch
 * allocations are; the kernels use 16-byte vector accesses and bulk copies).
 * Errors: QUAPI_ERR_ARG (n < 1, both outputs NULL, a misaligned pointer),
 * QUAPI_ERR_CUDA. */
quapi_status quapi_step_device(quapi_ctx* c, int64_t n, const void* A_in_dev, void* A_out_dev,
                               void* rho_dev);

/* Batched propagation of n independent contexts (one precision and one M for
 * all: FP64, FP32 or DF64; M = 2 or 3; each context in its own layout) to
 * their own final steps, in one persistent, CUDA-graph-captured launch.  The
 * library has no counterpart in the paper (which sweeps parameters one run at
 * a time); each instance's result equals its quapi_propagate result.
 *   ctxs[i]        contexts from quapi_setup / quapi_setup_eta (same precision, same M)
 *   rho0s[i]       [M*M] complex (host); Hermitian for a half-layout context
 *   nsteps_each[i] final step N_i >= 0
 *   rho_final[i]   [M*M] complex (host, caller-owned): rho(t_{N_i})
 * Work runs on ctxs[0]'s stream.  Blocks until all results are written.
 * Errors: QUAPI_ERR_ARG (NULL arrays, a context twice, N_i < 0, non-Hermitian
 * rho0 for a half-layout context), QUAPI_ERR_UNSUPPORTED (mixed precision or M),
 * QUAPI_ERR_TIMEOUT (a device-side dependency wait gave up), QUAPI_ERR_CUDA. */
quapi_status quapi_propagate_batch(int n, quapi_ctx* const* ctxs, const double* const* rho0s,
                                   const int64_t* nsteps_each, double* const* rho_final);

/* Copy the context's eta coefficients (4L+3 complex, layout of quapi_setup_eta). */
quapi_status quapi_get_eta(const quapi_ctx* c, double* eta_out);

/* Copy the context's U = exp(-i H dt) (M*M complex) and, if K_out is not NULL,
 * the pair propagator K (M^2 x M^2 complex, K[x'][x]). */
quapi_status quapi_get_propagator(const quapi_ctx* c, double* U_out, double* K_out);

/* Readout of rho(t_n) out of a caller's A_{n-1}, like quapi_step_device with
 * A_out_dev = NULL, but without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that must not touch the
 * CUDA allocator at that point, e.g. an application whose memory pool
 * already holds the free device memory (a raw cudaMalloc would fail), or a
 * time-critical loop that cannot afford cudaMalloc/cudaFree synchronising
 * the device.  The readout's per-CTA partial sums go to a fixed array inside
 * the library (216 KiB per device, kept until the process exits) instead of
 * the context's buffer.
 *   c          context from quapi_setup / quapi_setup_eta (its tables are used)
 *   n          >= 1: the path point whose rho(t_n) is read out
 *   A_in_dev   A_{n-1}: (M^2)^min(n,L) elements in the context's precision (device)
 *   rho_dev    M*M complex double (device), receives rho(t_n)
 * Asynchronous on the context's stream.  The device current at the call
 * must be the one that was current when the context was set up (the array's
 * address is per device).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one
 * array: calls whose kernels can overlap on the GPU (different streams, or
 * several host threads) race on it and must be serialised by the caller.
 * Errors: QUAPI_ERR_ARG (NULL pointers, n < 1, a pointer not 16-byte aligned,
 * M*M above the 9 partial sums a slot holds, a current device other than the
 * context's), QUAPI_ERR_CUDA. */
quapi_status quapi_readout_static(const quapi_ctx* c, int64_t n, const void* A_in_dev, void* rho_dev);

/* Number of kernels this library has launched in this process so far (all
 * contexts, all threads).  A diagnostic for benchmarks; never fails. */
uint64_t quapi_kernel_launches(void);

/* Description of the last error on c (or of the calling thread's last error
 * when c is NULL).  The string is owned by the library. */
const char* quapi_last_error(const quapi_ctx* c);

/* Release every resource of c (NULL is allowed). */
void quapi_destroy(quapi_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* QUAPI_H */
