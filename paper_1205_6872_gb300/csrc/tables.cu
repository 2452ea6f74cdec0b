// Setup kernels (FP64): the bare propagators, the initial tensor and the
// influence-functional factor tables of every tensor operation.
//
//  * propagator_kernel: U = exp(-i H dt) by scaling and squaring of a Taylor
//    series, then the pair propagator K(x', x) = U[a',a] conj(U[b',b]) -- the
//    forward and backward bare propagators of the path-integral expression
//    (Sec. II), x = a M + b.
//  * init_tensor_kernel: A_0(x) = rho0(x) exp(-d(x)(eta_00 s^+ - conj(eta_00) s^-)).
//  * build_tables_kernel: for one operation with n_in input digits, the
//    factor joining the new path point x to the point in input digit p is
//      G_p(x, x') = exp(-d(x) (eta_p s^+(x') - conj(eta_p) s^-(x')))   (Sec. II, Eq. for I)
//    times K(x, x') for the newest digit.  The kernel writes
//      isum[x][x']       = G_0                       (summed digit, if any)
//      lo[x][i]          = prod over the first j kept digits of G
//      hi[x][i]          = g(x) * prod over the remaining kept digits of G
//    with g(x) the self term of the new point, so that the propagator tensor
//    factor of a kept index is hi[x][i_hi] * lo[x][i_lo].  FP64 master values
//    are written as complex double (FP64 form) or split hi+lo floats (FP32 form).
#include <cmath>

#include "quapi_internal.h"

namespace quapi {

namespace {

constexpr int kMaxM = 4;

__device__ double2 cexp_d(double2 z) {
    double e = exp(z.x);
    double s, c;
    sincos(z.y, &s, &c);
    return make_double2(e * c, e * s);
}

__global__ void propagator_kernel(const double2* __restrict__ H, int M, double dt,
                                  double2* __restrict__ U_out, double2* __restrict__ K_out) {
    __shared__ double2 U[kMaxM * kMaxM];
    if (threadIdx.x == 0) {
        double2 A[kMaxM * kMaxM], T[kMaxM * kMaxM], term[kMaxM * kMaxM], tmp[kMaxM * kMaxM];
        // A = -i H dt
        for (int q = 0; q < M * M; ++q) A[q] = make_double2(H[q].y * dt, -H[q].x * dt);
        double norm = 0.0;
        for (int c = 0; c < M; ++c) {
            double col = 0.0;
            for (int r = 0; r < M; ++r) col += hypot(A[r * M + c].x, A[r * M + c].y);
            norm = fmax(norm, col);
        }
        int sq = 0;
        while (norm > 0.125 && sq < 60) {
            norm *= 0.5;
            ++sq;
        }
        double scale = ldexp(1.0, -sq);
        for (int q = 0; q < M * M; ++q) A[q] = make_double2(A[q].x * scale, A[q].y * scale);
        for (int r = 0; r < M; ++r)
            for (int c = 0; c < M; ++c) {
                T[r * M + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
                term[r * M + c] = T[r * M + c];
            }
        for (int k = 1; k <= 22; ++k) {  // ||A|| <= 1/8: remainder below 1e-40
            for (int r = 0; r < M; ++r)
                for (int c = 0; c < M; ++c) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int m = 0; m < M; ++m) acc = cfma(term[r * M + m], A[m * M + c], acc);
                    tmp[r * M + c] = make_double2(acc.x / k, acc.y / k);
                }
            for (int q = 0; q < M * M; ++q) {
                term[q] = tmp[q];
                T[q] = cadd(T[q], tmp[q]);
            }
        }
        for (int s = 0; s < sq; ++s) {
            for (int r = 0; r < M; ++r)
                for (int c = 0; c < M; ++c) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int m = 0; m < M; ++m) acc = cfma(T[r * M + m], T[m * M + c], acc);
                    tmp[r * M + c] = acc;
                }
            for (int q = 0; q < M * M; ++q) T[q] = tmp[q];
        }
        for (int q = 0; q < M * M; ++q) {
            U[q] = T[q];
            U_out[q] = T[q];
        }
    }
    __syncthreads();
    const int M2 = M * M;
    for (int e = threadIdx.x; e < M2 * M2; e += blockDim.x) {
        int xp = e / M2, x = e % M2;
        int ap = xp / M, bp = xp % M, a = x / M, b = x % M;
        K_out[e] = cmul(U[ap * M + a], cconj(U[bp * M + b]));
    }
}

__global__ void init_tensor_kernel(const double2* __restrict__ rho0, const double2* __restrict__ eta,
                                   int self0_idx, const double* __restrict__ s, int M, int form, int herm,
                                   void* A_out_base) {
    int x = threadIdx.x;
    if (x >= M * M) return;
    const int pos = x;  // one digit: the half layout stores every point too
    (void)herm;
    double sp = s[x / M], sm = s[x % M];
    double d = sp - sm;
    double2 e = eta[self0_idx];
    // -d (eta s^+ - conj(eta) s^-)
    double2 z = make_double2(-d * (e.x * sp - e.x * sm), -d * (e.y * sp + e.y * sm));
    double2 v = cmul(rho0[x], cexp_d(z));
    if (form == QUAPI_FP64) {
        reinterpret_cast<double2*>(A_out_base)[pos] = v;
    } else if (form == QUAPI_DF64) {
        df2 r;
        r.h = make_float2((float)v.x, (float)v.y);
        r.l = make_float2((float)(v.x - (double)r.h.x), (float)(v.y - (double)r.h.y));
        reinterpret_cast<df2*>(A_out_base)[pos] = r;
    } else {
        reinterpret_cast<float2*>(A_out_base)[pos] = make_float2((float)v.x, (float)v.y);
    }
}

__device__ __forceinline__ void store_entry(void* base, int64_t idx, int form, double2 v) {
    if (form == QUAPI_FP64) {
        reinterpret_cast<double2*>(base)[idx] = v;
    } else if (form == QUAPI_DF64) {
        // three floats per component: t1 + t2 + t3 reproduces the double v
        tf2 t;
        t.t1 = make_float2((float)v.x, (float)v.y);
        const double rx = v.x - (double)t.t1.x, ry = v.y - (double)t.t1.y;
        t.t2 = make_float2((float)rx, (float)ry);
        t.t3 = make_float2((float)(rx - (double)t.t2.x), (float)(ry - (double)t.t2.y));
        t.pad = make_float2(0.f, 0.f);
        reinterpret_cast<tf2*>(base)[idx] = t;
    } else {
        ff2 t;
        t.hr = (float)v.x;
        t.hi = (float)v.y;
        t.lr = (float)(v.x - (double)t.hr);
        t.li = (float)(v.y - (double)t.hi);
        reinterpret_cast<ff2*>(base)[idx] = t;
    }
}

constexpr int kBuildThreads = 256;
constexpr int kMaxM2 = 9;

__global__ void __launch_bounds__(kBuildThreads) build_tables_kernel(const BuildDesc* __restrict__ descs) {
    __shared__ double2 G[kMaxDigits][kMaxM2][kMaxM2];
    __shared__ double2 g[kMaxM2];
    const BuildDesc& D = descs[blockIdx.y];
    const int M = D.M, M2 = D.M2;
    // per-digit factor tables (one complex exponential each)
    for (int e = threadIdx.x; e < D.n_in * M2 * M2 + M2; e += blockDim.x) {
        if (e < D.n_in * M2 * M2) {
            int p = e / (M2 * M2), r = e % (M2 * M2);
            int x = r / M2, xp = r % M2;
            double d = D.s[x / M] - D.s[x % M];
            double spp = D.s[xp / M], smp = D.s[xp % M];
            double2 et = D.eta[D.eta_idx[p]];
            double2 z = make_double2(-d * (et.x * spp - et.x * smp), -d * (et.y * spp + et.y * smp));
            double2 v = (d == 0.0) ? make_double2(1.0, 0.0) : cexp_d(z);
            if (p == D.n_in - 1) v = cmul(v, D.K[x * M2 + xp]);
            G[p][x][xp] = v;
        } else {
            int x = e - D.n_in * M2 * M2;
            double sp = D.s[x / M], sm = D.s[x % M];
            double d = sp - sm;
            double2 et = D.eta[D.self_idx];
            double2 z = make_double2(-d * (et.x * sp - et.x * sm), -d * (et.y * sp + et.y * sm));
            g[x] = (d == 0.0) ? make_double2(1.0, 0.0) : cexp_d(z);
        }
    }
    __syncthreads();
    const int64_t n_isum = D.summed ? (int64_t)M2 * M2 : 0;
    const int64_t n_lo = (int64_t)M2 * D.lo_size;
    const int64_t n_hi = (int64_t)M2 * D.hi_size;
    const int64_t n_w = D.summed ? (int64_t)M2 * D.lo_size * M2 : 0;
    const int64_t total = n_isum + n_lo + n_hi + n_w;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n_isum) {
            int x = (int)(e / M2), xp = (int)(e % M2);
            store_entry(D.isum, e, D.form, G[0][x][xp]);
        } else if (e < n_isum + n_lo) {
            int64_t q = e - n_isum;
            int x = (int)(q / D.lo_size);
            int64_t i = q % D.lo_size;
            double2 v = make_double2(1.0, 0.0);
            for (int t = 0; t < D.j; ++t) {
                int digit = (int)(i % M2);
                i /= M2;
                v = cmul(v, G[D.summed + t][x][digit]);
            }
            store_entry(D.lo, q, D.form, v);
        } else if (e >= n_isum + n_lo + n_hi) {
            // w[x][f_lo][old] = (prod over the lo digits of G)(x, f_lo) * G_0(x, old)
            const int64_t q = e - n_isum - n_lo - n_hi;
            const int x = (int)(q / (D.lo_size * M2));
            const int64_t rem = q % (D.lo_size * M2);
            int64_t i = rem / M2;
            const int old = (int)(rem % M2);
            double2 v = G[0][x][old];
            for (int t = 0; t < D.j; ++t) {
                int digit = (int)(i % M2);
                i /= M2;
                v = cmul(v, G[D.summed + t][x][digit]);
            }
            store_entry(D.w, q, D.form, v);
        } else {
            int64_t q = e - n_isum - n_lo;
            int x = (int)(q / D.hi_size);
            int64_t i = q % D.hi_size;
            double2 v = g[x];
            for (int t = D.j; t < D.nk; ++t) {
                int digit = (int)(i % M2);
                i /= M2;
                v = cmul(v, G[D.summed + t][x][digit]);
            }
            store_entry(D.hi, q, D.form, v);
        }
    }
}

}  // namespace

cudaError_t launch_propagator(const double2* H_dev, int M, double dt, double2* U_dev, double2* K_dev,
                              cudaStream_t st) {
    if (M < 1 || M > kMaxM) return cudaErrorInvalidValue;
    propagator_kernel<<<1, 128, 0, st>>>(H_dev, M, dt, U_dev, K_dev);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init_tensor(const double2* rho0_dev, const double2* eta, int self0_idx,
                               const double* s, int M, int form, void* A_out, cudaStream_t st, int herm) {
    init_tensor_kernel<<<1, 32, 0, st>>>(rho0_dev, eta, self0_idx, s, M, form, herm, A_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_build_tables(const BuildDesc* descs_dev, int ndesc, int /*M2*/, int64_t max_entries,
                                cudaStream_t st) {
    if (ndesc <= 0) return cudaSuccess;
    int64_t blocks = (max_entries + kBuildThreads - 1) / kBuildThreads;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    dim3 grid((unsigned)blocks, (unsigned)ndesc);
    build_tables_kernel<<<grid, kBuildThreads, 0, st>>>(descs_dev);
    count_launch();
    return cudaGetLastError();
}

}  // namespace quapi
