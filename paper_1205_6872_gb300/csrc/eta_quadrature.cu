// eta quadrature (FP64 on the GPU).
//
// The eta coefficients (Sec. II, Eqs. etaKK'generalTrotter .. etaNkgeneralStrang)
// are double integrals of the bath response function
//   alpha(t) = (1/pi) int_0^inf J(w) [coth(beta w/2) cos(w t) - i sin(w t)] dw
// (Eq. bathResponseFunction) over the time boxes of two path points.  Doing
// the time integrals first leaves one frequency integral per eta:
//   disjoint boxes (widths w1 later, w2 earlier, centres D apart):
//     (1/pi) int J/w^2 4 sin(w w1/2) sin(w w2/2) [coth(beta w/2) cos(w D) - i sin(w D)] dw
//   a box of width w with itself (inner time below the outer one):
//     (1/pi) int J/w^2 [coth(beta w/2) (1 - cos w w) + i (sin w w - w w)] dw
// Each is evaluated with a composite Gauss-Legendre rule (16 nodes per panel)
// on [0, w_max]; one CTA per eta, FP64 accumulation, fixed-order reduction.
// A tabulated J (piecewise linear) gets panels that never straddle a table
// node, so the rule sees a smooth integrand on every panel.
#include <cmath>
#include <vector>

#include "quapi_internal.h"

namespace quapi {

namespace {

constexpr int kEtaThreads = 256;
constexpr int kMaxGL = 32;

__device__ __forceinline__ double j_over_w2(int kind, double a, double wc, double w) {
    if (kind == QUAPI_J_OHMIC_EXP) return 1.5707963267948966 * a * exp(-w / wc) / w;
    double r = w / wc;
    return a * w * exp(-r * r);
}

// sin(x) - x: odd Taylor series for |x| < 1 (terms to x^23), direct difference otherwise.
__device__ __forceinline__ double sin_minus_x(double x) {
    if (fabs(x) >= 1.0) return sin(x) - x;
    double x2 = x * x;
    double term = -x * x2 / 6.0;
    double acc = term;
#pragma unroll
    for (int k = 2; k <= 11; ++k) {
        term = -term * x2 / double((2 * k) * (2 * k + 1));
        acc += term;
    }
    return acc;
}

// One quadrature node: adds (1/pi) wt J(w)/w^2 times the box kernel of job jb at frequency w.
__device__ __forceinline__ void eta_node(const EtaJob& jb, double beta, double w, double jw, double& acc_re,
                                         double& acc_im) {
    const double cth = 1.0 / tanh(0.5 * beta * w);
    if (jb.w2 < 0.0) {  // self box
        const double sh = sin(0.5 * w * jb.w1);
        acc_re += jw * cth * 2.0 * sh * sh;
        acc_im += jw * sin_minus_x(w * jb.w1);
    } else {
        const double c = jw * 4.0 * sin(0.5 * w * jb.w1) * sin(0.5 * w * jb.w2);
        double sd, cd;
        sincos(w * jb.D, &sd, &cd);
        acc_re += c * cth * cd;
        acc_im -= c * sd;
    }
}

// Fixed-order block reduction of the two accumulators into out.
__device__ __forceinline__ void eta_reduce(double acc_re, double acc_im, double2* out) {
    __shared__ double red_re[kEtaThreads / 32], red_im[kEtaThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc_re += __shfl_down_sync(0xffffffffu, acc_re, off);
        acc_im += __shfl_down_sync(0xffffffffu, acc_im, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red_re[warp] = acc_re;
        red_im[warp] = acc_im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0, m = 0.0;
        for (int k = 0; k < kEtaThreads / 32; ++k) {
            r += red_re[k];
            m += red_im[k];
        }
        *out = make_double2(r, m);
    }
}

// Tabulated J: panels [pw[p], pw[p+1]] each inside one segment of the table, J linear on the
// panel between its end values pj[p], pj[p+1].
__global__ void __launch_bounds__(kEtaThreads) eta_kernel_tab(const EtaJob* __restrict__ jobs, double beta,
                                                              const double* __restrict__ pw,
                                                              const double* __restrict__ pj, int panels,
                                                              const double* __restrict__ gl, int gl_n,
                                                              double2* __restrict__ out) {
    __shared__ double sx[kMaxGL], sw[kMaxGL];
    if (threadIdx.x < gl_n) {
        sx[threadIdx.x] = gl[threadIdx.x];
        sw[threadIdx.x] = gl[gl_n + threadIdx.x];
    }
    __syncthreads();
    const EtaJob jb = jobs[blockIdx.x];
    const double inv_pi = 0.31830988618379067;
    double acc_re = 0.0, acc_im = 0.0;
    const int64_t nodes = (int64_t)panels * gl_n;
    for (int64_t q = threadIdx.x; q < nodes; q += kEtaThreads) {
        const int panel = (int)(q / gl_n);
        const int i = (int)(q - (int64_t)panel * gl_n);
        const double lo = pw[panel], h = pw[panel + 1] - lo;
        const double t = 0.5 * (1.0 + sx[i]);
        const double w = lo + h * t;
        const double J = pj[panel] + (pj[panel + 1] - pj[panel]) * t;
        eta_node(jb, beta, w, J / (w * w) * inv_pi * (0.5 * h * sw[i]), acc_re, acc_im);
    }
    eta_reduce(acc_re, acc_im, out + blockIdx.x);
}

__global__ void __launch_bounds__(kEtaThreads) eta_kernel(const EtaJob* __restrict__ jobs, int kind,
                                                          double a, double wc, double beta,
                                                          double wmax, int panels,
                                                          const double* __restrict__ gl, int gl_n,
                                                          double2* __restrict__ out) {
    __shared__ double sx[kMaxGL], sw[kMaxGL];
    if (threadIdx.x < gl_n) {
        sx[threadIdx.x] = gl[threadIdx.x];
        sw[threadIdx.x] = gl[gl_n + threadIdx.x];
    }
    __syncthreads();
    const EtaJob jb = jobs[blockIdx.x];
    const double h = wmax / panels;
    const double inv_pi = 0.31830988618379067;
    double acc_re = 0.0, acc_im = 0.0;
    const int64_t nodes = (int64_t)panels * gl_n;
    for (int64_t q = threadIdx.x; q < nodes; q += kEtaThreads) {
        const int panel = (int)(q / gl_n);
        const int i = (int)(q - (int64_t)panel * gl_n);
        const double w = h * (panel + 0.5 * (1.0 + sx[i]));
        eta_node(jb, beta, w, j_over_w2(kind, a, wc, w) * inv_pi * (0.5 * h * sw[i]), acc_re, acc_im);
    }
    eta_reduce(acc_re, acc_im, out + blockIdx.x);
}

}  // namespace

// n-point Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on
// P_n (three-term recurrence for P_n and its derivative).
void gauss_legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

cudaError_t launch_eta_quadrature(const EtaJob* jobs_dev, int njobs, int kind, double a, double wc,
                                  double beta, int panels, const double* gl_dev, int gl_n,
                                  double2* eta_out, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    if (gl_n > kMaxGL) return cudaErrorInvalidValue;
    double wmax = (kind == QUAPI_J_OHMIC_EXP) ? 46.0 * wc : 7.5 * wc;
    eta_kernel<<<njobs, kEtaThreads, 0, st>>>(jobs_dev, kind, a, wc, beta, wmax, panels, gl_dev, gl_n,
                                              eta_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eta_quadrature_tab(const EtaJob* jobs_dev, int njobs, double beta, const double* pw_dev,
                                      const double* pj_dev, int panels, const double* gl_dev, int gl_n,
                                      double2* eta_out, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    if (gl_n > kMaxGL || panels < 1) return cudaErrorInvalidValue;
    eta_kernel_tab<<<njobs, kEtaThreads, 0, st>>>(jobs_dev, beta, pw_dev, pj_dev, panels, gl_dev, gl_n, eta_out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace quapi
