/* Plain FP64 loops of the tensor-propagator recurrence -- TEST INFRASTRUCTURE ONLY.
 *
 * Part of the CPU oracle.  It shares nothing with the CUDA library.  Every
 * function evaluates, element by element, one application of the propagator
 * tensor T = K * prod I_dk (Sec. I: Makri-Makarov tensor propagator scheme;
 * Sec. II: path-integral expression and discretised influence functional) to
 * the augmented tensor A.
 *
 * Conventions.  M2 = M*M values per path point.  A tensor with n digits is a
 * flat array of M2^n complex numbers; digit p (p = 0 least significant) of the
 * flat index holds one path point, the oldest point in digit 0.  The caller
 * supplies, per digit p, the factor table G[p][x_new][x] coupling the new path
 * point x_new to the point stored in digit p (the bare propagator K is already
 * folded into the table of the newest digit), and g[x_new], the self factor
 * of the new point.  All arrays are interleaved (re, im) doubles.
 *
 *   oracle_grow    : out[x_new * M2^n + i] = g[x_new] * prod_p G[p][x_new][d_p(i)] * A[i]
 *   oracle_step    : out[x_new * M2^(n-1) + f] =
 *                      g[x_new] * prod_{p>=1} G[p][x_new][d_p] * sum_{d_0} G[0][x_new][d_0] * A[f*M2 + d_0]
 *                    (multiply by T, then sum over the oldest path index)
 *   oracle_readout : rho[x_new] = sum over every digit of the same product
 *
 * Factors that do not depend on the summed digit are multiplied outside the
 * inner sum; nothing else is reordered.  OpenMP splits the output elements;
 * the readout sums fixed chunks and then adds the chunk sums in order, so its
 * result does not depend on the thread count.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>

typedef double complex cplx;

static int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

static cplx kept_product(int M2, int n, int p_first, const cplx* G, const cplx* g,
                         int xn, int64_t index_of_digit0) {
    /* g[xn] * prod_{p = p_first}^{n-1} G[p][xn][digit_p(index)] */
    cplx prod = g[xn];
    int64_t rest = index_of_digit0;
    for (int p = 0; p < n; ++p) {
        int digit = (int)(rest % M2);
        rest /= M2;
        if (p >= p_first) prod *= G[((int64_t)p * M2 + xn) * M2 + digit];
    }
    return prod;
}

void oracle_grow(int M2, int n, const double* A_in, const double* Gd, const double* gd,
                 double* A_out) {
    const cplx* A = (const cplx*)A_in;
    const cplx* G = (const cplx*)Gd;
    const cplx* g = (const cplx*)gd;
    cplx* out = (cplx*)A_out;
    int64_t S = ipow(M2, n);
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < (int64_t)M2 * S; ++o) {
        int xn = (int)(o / S);
        int64_t i = o % S;
        out[o] = kept_product(M2, n, 0, G, g, xn, i) * A[i];
    }
}

void oracle_step(int M2, int n, const double* A_in, const double* Gd, const double* gd,
                 double* A_out) {
    const cplx* A = (const cplx*)A_in;
    const cplx* G = (const cplx*)Gd;
    const cplx* g = (const cplx*)gd;
    cplx* out = (cplx*)A_out;
    int64_t F = ipow(M2, n - 1);
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < (int64_t)M2 * F; ++o) {
        int xn = (int)(o / F);
        int64_t f = o % F;
        cplx sum = 0.0;
        for (int d0 = 0; d0 < M2; ++d0)
            sum += G[((int64_t)0 * M2 + xn) * M2 + d0] * A[f * M2 + d0];
        out[o] = kept_product(M2, n, 1, G, g, xn, f * M2) * sum;
    }
}

void oracle_readout(int M2, int n, const double* A_in, const double* Gd, const double* gd,
                    double* rho_out) {
    const cplx* A = (const cplx*)A_in;
    const cplx* G = (const cplx*)Gd;
    const cplx* g = (const cplx*)gd;
    int64_t F = ipow(M2, n - 1);
    const int64_t chunk = 4096;
    int64_t nchunks = (F + chunk - 1) / chunk;
    cplx* part = (cplx*)calloc((size_t)(nchunks * M2), sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nchunks; ++c) {
        int64_t f_end = (c + 1) * chunk < F ? (c + 1) * chunk : F;
        for (int xn = 0; xn < M2; ++xn) {
            cplx acc = 0.0;
            for (int64_t f = c * chunk; f < f_end; ++f) {
                cplx sum = 0.0;
                for (int d0 = 0; d0 < M2; ++d0)
                    sum += G[((int64_t)0 * M2 + xn) * M2 + d0] * A[f * M2 + d0];
                acc += kept_product(M2, n, 1, G, g, xn, f * M2) * sum;
            }
            part[c * M2 + xn] = acc;
        }
    }
    cplx* rho = (cplx*)rho_out;
    for (int xn = 0; xn < M2; ++xn) {
        cplx acc = 0.0;
        for (int64_t c = 0; c < nchunks; ++c) acc += part[c * M2 + xn];
        rho[xn] = acc;
    }
    free(part);
}
