// Device code shared by the MCG sweep kernels (FP64 in mcg_sweep.cu, compact
// FP32 in mcg_sweep_f32.cu): the exact local maximisation of the SU(2)
// subgroup problem (Jacobi eigen-decomposition + secular equation, Newton on
// the KKT system with an LDL^T positivity certificate), the per-warp R
// partial sums and the block -> field map of a batch.  Included by each sweep
// translation unit (whole-program device compilation: every unit keeps its
// own copy).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "mcg_common.cuh"
#include "mcg_internal.h"

namespace mcg {

// ---------------------------------------------------------------------------
// 4x4 symmetric eigen-decomposition (cyclic Jacobi)
// ---------------------------------------------------------------------------
// FP32 solves use the SFU approximations (rsqrt, reciprocal: ~1-2 ulp); the
// FP64 fallback path uses IEEE operations.
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }

template <typename T, int P, int Q>
__device__ __forceinline__ void jrot(T (&S)[4][4], T (&V)[4][4]) {
    const T apq = S[P][Q];
    const T th = (S[Q][Q] - S[P][P]) * T(0.5);
    const T den = fabs(th) + fsqrt(th * th + apq * apq);
    T t = den > T(0) ? apq * frcp(den) : T(0);
    if (th < T(0)) t = -t;
    const T c = rsqrt(T(1) + t * t);
    const T s = t * c;
    S[P][P] -= t * apq;
    S[Q][Q] += t * apq;
    S[P][Q] = T(0);
    S[Q][P] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == P || k == Q) continue;
        const T akp = S[k][P], akq = S[k][Q];
        const T np = c * akp - s * akq, nq = s * akp + c * akq;
        S[k][P] = np;
        S[P][k] = np;
        S[k][Q] = nq;
        S[Q][k] = nq;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T vkp = V[k][P], vkq = V[k][Q];
        V[k][P] = c * vkp - s * vkq;
        V[k][Q] = s * vkp + c * vkq;
    }
}

template <typename T>
__device__ __forceinline__ void jacobi4(T (&S)[4][4], T (&V)[4][4], int max_sweeps, T rel_tol) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) V[i][j] = (i == j) ? T(1) : T(0);
    T fro2 = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fro2 += S[i][j] * S[i][j];
#pragma unroll 1
    for (int sw = 0; sw < max_sweeps; ++sw) {
        const T off = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[0][3] * S[0][3] + S[1][2] * S[1][2] +
                      S[1][3] * S[1][3] + S[2][3] * S[2][3];
        if (off <= rel_tol * rel_tol * fro2) break;
        jrot<T, 0, 1>(S, V);
        jrot<T, 0, 2>(S, V);
        jrot<T, 0, 3>(S, V);
        jrot<T, 1, 2>(S, V);
        jrot<T, 1, 3>(S, V);
        jrot<T, 2, 3>(S, V);
    }
}

// Trust-region maximiser from the eigen-decomposition (al, V columns).
// Returns 0 easy case, 1 hard case.  mu_out is the multiplier.
// The secular equation n(d) = 1, n(d)^2 = sum_i beta_i^2 / (d + g_i)^2, is
// solved for the offset d = mu - al_max > 0 with g_i = al_max - al_i (0 on the
// top eigenspace), so that d keeps its relative precision when it is tiny (a
// weight beta_top near zero: near the hard case).  Newton on 1/n(d) - 1, which
// is concave and increasing in d (the Moré-Sorensen form), climbs
// monotonically to the root from any point where n >= 1: from d = |beta_top|,
// or, when the other eigendirections alone have n >= 1 at d = 0 (then the
// root lies beyond theirs), from the root of their equation, solved first the
// same way.  Without that start a tiny beta_top makes every step tiny.
template <typename T>
__device__ __forceinline__ int trs_from_eigen(const T (&S)[4][4], const T (&V)[4][4], const T (&b)[4], T (&a)[4],
                                              T& mu_out) {
    const T eps = sizeof(T) == 8 ? T(2.2e-16) : T(1.2e-7);
    const T deg_tol = sizeof(T) == 8 ? T(1e-13) : T(1e-5);
    const T hard_tol = sizeof(T) == 8 ? T(1e-14) : T(1e-6);
    T al[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) al[i] = S[i][i];
    const T bn = fsqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
    T scale = bn;
#pragma unroll
    for (int i = 0; i < 4; ++i) scale = fmax(scale, fabs(al[i]));
    if (scale == T(0)) {
        a[0] = T(1);
        a[1] = a[2] = a[3] = T(0);
        mu_out = T(0);
        return 1;
    }
    T amax = al[0];
    int imax = 0;
#pragma unroll
    for (int i = 1; i < 4; ++i)
        if (al[i] > amax) {
            amax = al[i];
            imax = i;
        }
    T beta[4], gap[4];
    T btop2 = T(0), pn2 = T(0);
    bool top[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        beta[i] = V[0][i] * b[0] + V[1][i] * b[1] + V[2][i] * b[2] + V[3][i] * b[3];
        gap[i] = amax - al[i];
        top[i] = gap[i] <= deg_tol * scale;
        if (top[i]) {
            gap[i] = T(0);
            btop2 += beta[i] * beta[i];
        } else {
            const T c = fdiv(beta[i], gap[i]);
            pn2 += c * c;
        }
    }
    const T btop = fsqrt(btop2);
    if (btop <= hard_tol * scale && pn2 < T(1)) {
        // hard case: the partial solution plus the top eigenvector, its
        // largest component positive, filling the unit norm
        T vm[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            vm[k] = V[k][0];
#pragma unroll
            for (int i = 1; i < 4; ++i)
                if (i == imax) vm[k] = V[k][i];
        }
        int kb = 0;
        T vb = fabs(vm[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (fabs(vm[k]) > vb) {
                vb = fabs(vm[k]);
                kb = k;
            }
        T sgn = T(1);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k == kb) sgn = vm[k] >= T(0) ? T(1) : T(-1);
        const T t = fsqrt(T(1) - pn2) * sgn;
        T coef[4], n2 = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) coef[i] = top[i] ? T(0) : fdiv(beta[i], gap[i]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = V[k][0] * coef[0] + V[k][1] * coef[1] + V[k][2] * coef[2] + V[k][3] * coef[3] + t * vm[k];
            n2 += a[k] * a[k];
        }
        const T inv = rsqrt(n2);
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] *= inv;
        mu_out = amax;
        return 1;
    }
    const int maxit = sizeof(T) == 8 ? 100 : 40;
    // easy case: the root d lies in [btop, bn] (n >= 1 at btop from the top
    // weights alone, n <= 1 at bn)
    T lo = btop, hi = bn, d = btop;
    if (pn2 >= T(1)) {
        T dr = T(0);
#pragma unroll 1
        for (int it = 0; it < maxit; ++it) {
            T s2 = T(0), s3 = T(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (top[i]) continue;
                const T r = frcp(dr + gap[i]);
                const T q = beta[i] * beta[i] * r * r;
                s2 += q;
                s3 += q * r;
            }
            if (!(s3 > T(0))) break;
            const T step = fdiv((fsqrt(s2) - T(1)) * s2, s3);
            dr += step;
            if (!(step > T(4) * eps * dr)) break;
        }
        d = fmax(d, fmin(dr, hi));
    }
#pragma unroll 1
    for (int it = 0; it < maxit; ++it) {
        T s2 = T(0), s3 = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // a zero weight contributes nothing (also where d + gap is 0)
            if (beta[i] == T(0)) continue;
            const T r = frcp(d + gap[i]);
            const T q = beta[i] * beta[i] * r * r;
            s2 += q;
            s3 += q * r;
        }
        const T n = fsqrt(s2);
        if (n >= T(1))
            lo = fmax(lo, d);
        else
            hi = fmin(hi, d);
        T next = d + fdiv((n - T(1)) * s2, s3);
        if (!(next > lo && next < hi)) next = T(0.5) * (lo + hi);
        if (fabs(next - d) <= T(4) * eps * d) {
            d = next;
            break;
        }
        d = next;
        if (hi - lo <= T(4) * eps * d) break;
    }
    T n2 = T(0);
    T coef[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) coef[i] = beta[i] == T(0) ? T(0) : fdiv(beta[i], d + gap[i]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = V[k][0] * coef[0] + V[k][1] * coef[1] + V[k][2] * coef[2] + V[k][3] * coef[3];
        n2 += a[k] * a[k];
    }
    const T inv = rsqrt(n2);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] *= inv;
    mu_out = amax + d;
    return 0;
}

// ---------------------------------------------------------------------------
// Newton on the KKT system from a warm start, certified by LDL^T
// ---------------------------------------------------------------------------
// LDL^T of the symmetric 4x4 matrix M (no pivoting).  Returns the smallest
// pivot relative to the largest in absolute value (negative if M is not
// positive definite); Dinv receives the inverse pivots.
template <typename T>
__device__ __forceinline__ T ldlt4(const T (&M)[4][4], T (&L)[4][4], T (&Dinv)[4]) {
    T D[4];
    D[0] = M[0][0];
    Dinv[0] = frcp(D[0]);
    L[1][0] = M[1][0] * Dinv[0];
    L[2][0] = M[2][0] * Dinv[0];
    L[3][0] = M[3][0] * Dinv[0];
    D[1] = M[1][1] - L[1][0] * L[1][0] * D[0];
    Dinv[1] = frcp(D[1]);
    L[2][1] = (M[2][1] - L[2][0] * L[1][0] * D[0]) * Dinv[1];
    L[3][1] = (M[3][1] - L[3][0] * L[1][0] * D[0]) * Dinv[1];
    D[2] = M[2][2] - L[2][0] * L[2][0] * D[0] - L[2][1] * L[2][1] * D[1];
    Dinv[2] = frcp(D[2]);
    L[3][2] = (M[3][2] - L[3][0] * L[2][0] * D[0] - L[3][1] * L[2][1] * D[1]) * Dinv[2];
    D[3] = M[3][3] - L[3][0] * L[3][0] * D[0] - L[3][1] * L[3][1] * D[1] - L[3][2] * L[3][2] * D[2];
    Dinv[3] = frcp(D[3]);
    T dmin = fmin(fmin(D[0], D[1]), fmin(D[2], D[3]));
    T dmax = fmax(fmax(fabs(D[0]), fabs(D[1])), fmax(fabs(D[2]), fabs(D[3])));
    return dmax > T(0) ? fdiv(dmin, dmax) : T(-1);
}

template <typename T, typename U>
__device__ __forceinline__ void ldlt4_solve(const T (&L)[4][4], const T (&Dinv)[4], const U (&r)[4], T (&x)[4]) {
    T z0 = (T)r[0];
    T z1 = (T)r[1] - L[1][0] * z0;
    T z2 = (T)r[2] - L[2][0] * z0 - L[2][1] * z1;
    T z3 = (T)r[3] - L[3][0] * z0 - L[3][1] * z1 - L[3][2] * z2;
    z0 *= Dinv[0];
    z1 *= Dinv[1];
    z2 *= Dinv[2];
    z3 *= Dinv[3];
    x[3] = z3;
    x[2] = z2 - L[3][2] * x[3];
    x[1] = z1 - L[2][1] * x[2] - L[3][1] * x[3];
    x[0] = z0 - L[1][0] * x[1] - L[2][0] * x[2] - L[3][0] * x[3];
}

// Newton iterations on (mu - A) a = b, |a| = 1 starting from a = (1,0,0,0)
// (the current links, i.e. no change) with mu its Lagrange estimate.  On
// convergence returns true with a normalised, mu, and the LDL^T factors of
// (mu_f - A), mu_f the multiplier of the last factorisation (mu = mu_f plus
// the last step), with pd its smallest pivot relative to the largest.  That mu
// is above lambda_max(A) (a the global maximum of the trust-region
// subproblem) is for the caller to certify: see above_lambda_max.
template <typename T>
__device__ __forceinline__ bool kkt_newton(const T (&A)[4][4], const T (&b)[4], T (&a)[4], T& mu, T (&L)[4][4],
                                           T (&Dinv)[4], T& pd, T& mu_f) {
    const T conv = sizeof(T) == 8 ? T(1e-13) : T(2e-6);
    a[0] = T(1);
    a[1] = a[2] = a[3] = T(0);
    mu = A[0][0] + b[0];
    mu_f = mu;
    bool ok = false;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        mu_f = mu;
        T M[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) M[i][j] = (i == j ? mu : T(0)) - A[i][j];
        pd = ldlt4(M, L, Dinv);
        if (!(fabs(pd) > T(1e-12))) return false;  // singular or NaN
        T r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = b[k] - (M[k][0] * a[0] + M[k][1] * a[1] + M[k][2] * a[2] + M[k][3] * a[3]);
        const T sres = T(0.5) * (T(1) - (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]));
        T x[4], y[4];
        ldlt4_solve(L, Dinv, r, x);
        ldlt4_solve(L, Dinv, a, y);
        const T ay = a[0] * y[0] + a[1] * y[1] + a[2] * y[2] + a[3] * y[3];
        const T dmu = fdiv(a[0] * x[0] + a[1] * x[1] + a[2] * x[2] + a[3] * x[3] - sres, ay);
        T dmax = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T da = x[k] - dmu * y[k];
            a[k] += da;
            dmax = fmax(dmax, fabs(da));
        }
        mu += dmu;
        if (dmax <= conv) {
            ok = true;
            break;
        }
    }
    if (!ok) return false;
    const T inv = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] *= inv;
    return pd > (sizeof(T) == 8 ? T(1e-12) : T(1e-5));
}

// Certificate that a multiplier mu lies above lambda_max(A) by more than
// margin times the trace of mu_f - A, given the inverse pivots Dinv of the
// LDL^T of the positive definite matrix mu_f - A: its smallest eigenvalue is
// at least 27 det / tr^3 (det the product of the pivots, tr the trace; the
// other three eigenvalues have a product of at most (tr / 3)^3), so
// lambda_max(A) <= mu_f - 27 det / tr^3.
template <typename T>
__device__ __forceinline__ bool above_lambda_max(const T (&A)[4][4], const T (&Dinv)[4], T mu_f, double mu,
                                                 double margin) {
    const double det = 1.0 / (((double)Dinv[0] * (double)Dinv[1]) * ((double)Dinv[2] * (double)Dinv[3]));
    const double tr = (((double)mu_f - A[0][0]) + ((double)mu_f - A[1][1])) +
                      (((double)mu_f - A[2][2]) + ((double)mu_f - A[3][3]));
    return (mu - (double)mu_f) + 27.0 * det / (tr * tr * tr) > margin * tr;
}

// FP32 solve of the subproblem given A (symmetric) and b (Jacobi + secular;
// out of line: the warm-started Newton path handles almost every solve).
static __device__ __noinline__ int solve_f32(const float (&A)[4][4], const float (&b)[4], float (&a)[4], float& mu,
                                         float (&S)[4][4], float (&V)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) S[i][j] = A[i][j];
    jacobi4<float>(S, V, 8, 5e-7f);
    return trs_from_eigen<float>(S, V, b, a, mu);
}

// Newton refinement of (a, mu) on the KKT system (mu - A) a = b, |a| = 1.
// Residuals are evaluated in FP64; the correction uses the FP32
// eigen-decomposition (S diagonal, V) at the FP32 multiplier as a fixed
// approximate inverse of (mu - A), so each step contracts the error by about
// cond(mu - A) * 1e-7.  Stops once the correction is below 1e-12 (the next one
// would be below FP64 resolution).  Returns false if that does not happen in
// 6 steps.
__device__ __forceinline__ bool kkt_refine(const double (&A)[4][4], const double (&b)[4], const float (&S)[4][4],
                                           const float (&V)[4][4], const float (&af)[4], float muf, double (&a)[4],
                                           double& mu) {
    float d[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = __fdividef(1.0f, muf - S[i][i]);
    float at[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) at[i] = (V[0][i] * af[0] + V[1][i] * af[1] + V[2][i] * af[2] + V[3][i] * af[3]) * d[i];
    double y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        y[k] = (double)(V[k][0] * at[0] + V[k][1] * at[1] + V[k][2] * at[2] + V[k][3] * at[3]);
        a[k] = (double)af[k];
    }
    mu = (double)muf;
    const double inv_ay = 1.0 / (a[0] * y[0] + a[1] * y[1] + a[2] * y[2] + a[3] * y[3]);
#pragma unroll 1
    for (int it = 0; it < 6; ++it) {
        float rf[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double acc = fma(-mu, a[k], b[k]);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc = fma(A[k][j], a[j], acc);
            rf[k] = (float)acc;
        }
        const double s = 0.5 * (1.0 - (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]));
        float rt[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) rt[i] = (V[0][i] * rf[0] + V[1][i] * rf[1] + V[2][i] * rf[2] + V[3][i] * rf[3]) * d[i];
        double x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = (double)(V[k][0] * rt[0] + V[k][1] * rt[1] + V[k][2] * rt[2] + V[k][3] * rt[3]);
        const double dmu = (a[0] * x[0] + a[1] * x[1] + a[2] * x[2] + a[3] * x[3] - s) * inv_ay;
        double dmax = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double da = fma(-dmu, y[k], x[k]);
            a[k] += da;
            dmax = fmax(dmax, fabs(da));
        }
        mu += dmu;
        if (!(dmax == dmax)) return false;  // NaN
        if (dmax <= 1e-12) return true;
    }
    return false;
}

// Full FP64 solve (Jacobi + secular), kept out of line: it runs only for the
// rare local problems the refinement cannot settle.
static __device__ __noinline__ void solve_f64_full(const double* Ain, const double* b_in, double* a_out) {
    double Sd[4][4], Vd[4][4], bd[4], ad[4], mud;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bd[i] = b_in[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) Sd[i][j] = Ain[4 * i + j];
    }
    jacobi4<double>(Sd, Vd, 30, 1e-15);
    trs_from_eigen<double>(Sd, Vd, bd, ad, mud);
#pragma unroll
    for (int k = 0; k < 4; ++k) a_out[k] = ad[k];
}

template <typename T>
struct Solver;

// FP64 refinement with the FP32 LDL^T factors of (mu32 - A) as the fixed
// approximate inverse (same iteration as kkt_refine).
__device__ __forceinline__ bool kkt_refine_ldlt(const double (&A)[4][4], const double (&b)[4], const float (&L)[4][4],
                                                const float (&Dinv)[4], const float (&af)[4], float muf, double (&a)[4],
                                                double& mu_out) {
    float yf[4];
    ldlt4_solve(L, Dinv, af, yf);
    double y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        y[k] = (double)yf[k];
        a[k] = (double)af[k];
    }
    double mu = (double)muf;
    const double inv_ay = 1.0 / (a[0] * y[0] + a[1] * y[1] + a[2] * y[2] + a[3] * y[3]);
#pragma unroll 1
    for (int it = 0; it < 6; ++it) {
        float rf[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double acc = fma(-mu, a[k], b[k]);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc = fma(A[k][j], a[j], acc);
            rf[k] = (float)acc;
        }
        const double s = 0.5 * (1.0 - (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]));
        float xf[4];
        ldlt4_solve(L, Dinv, rf, xf);
        double x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = (double)xf[k];
        const double dmu = (a[0] * x[0] + a[1] * x[1] + a[2] * x[2] + a[3] * x[3] - s) * inv_ay;
        double dmax = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double da = fma(-dmu, y[k], x[k]);
            a[k] += da;
            dmax = fmax(dmax, fabs(da));
        }
        mu += dmu;
        mu_out = mu;
        if (!(dmax == dmax)) return false;
        if (dmax <= 1e-12) return true;
    }
    return false;
}

struct Vec4d {
    double v[4];
};

// The rare FP64 local solves the warm-started path cannot settle: FP32 Jacobi
// + secular seed refined in FP64 (kkt_refine), else the full FP64 Jacobi +
// secular solve.  Out of line with A and b passed by value, so the caller's
// copies stay in registers; the result is normalised.
static __device__ __noinline__ Vec4d solve_f64_fallback(double a00, double a01, double a02, double a03, double a11,
                                                 double a12, double a13, double a22, double a23, double a33,
                                                 double b0, double b1, double b2, double b3) {
    const double A[4][4] = {{a00, a01, a02, a03}, {a01, a11, a12, a13}, {a02, a12, a22, a23}, {a03, a13, a23, a33}};
    const double b[4] = {b0, b1, b2, b3};
    float Af[4][4], bf[4], af[4], muf;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bf[i] = (float)b[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) Af[i][j] = (float)A[i][j];
    }
    Vec4d r;
    bool ok = false;
    float S[4][4], V[4][4];
    const int hard = solve_f32(Af, bf, af, muf, S, V);
    if (!hard) {
        float amax = S[0][0], amin = S[0][0];
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            amax = fmaxf(amax, S[i][i]);
            amin = fminf(amin, S[i][i]);
        }
        const float gap = muf - amax;
        if (gap > 2e-4f * (muf - amin + 1e-30f)) {
            double mu;
            ok = kkt_refine(A, b, S, V, af, muf, r.v, mu);
        }
    }
    if (!ok) {
        double Aflat[16];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Aflat[4 * i + j] = A[i][j];
        solve_f64_full(Aflat, b, r.v);
        if (!(isfinite(r.v[0]) && isfinite(r.v[1]) && isfinite(r.v[2]) && isfinite(r.v[3]))) {
            r.v[0] = 1.0;  // backstop: the identity leaves the site unchanged
            r.v[1] = r.v[2] = r.v[3] = 0.0;
        }
        return r;
    }
    const double inv = rsqrt(r.v[0] * r.v[0] + r.v[1] * r.v[1] + r.v[2] * r.v[2] + r.v[3] * r.v[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) r.v[k] *= inv;
    return r;
}

template <>
struct Solver<double> {
    // returns 1 when the warm-started path did not settle the problem
    __device__ __forceinline__ static int solve(const double (&A)[4][4], const double (&b)[4], double (&a)[4]) {
        float Af[4][4], bf[4], af[4], muf;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            bf[i] = (float)b[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) Af[i][j] = (float)A[i][j];
        }
        bool ok = false;
        {
            float L[4][4], Dinv[4], pd, mu_f;
            // warm-started FP32 Newton; the refinement contracts by ~cond * 1e-7,
            // with cond ~ 1 / pd bounded by the pivot test.  Certificate: the
            // refined multiplier above lambda_max of the FP32 copy of A by 1e-6
            // of the trace of mu_f - A (far above the FP32 rounding of A)
            double mu = 0.0;
            if (kkt_newton<float>(Af, bf, af, muf, L, Dinv, pd, mu_f) && pd > 2e-4f)
                ok = kkt_refine_ldlt(A, b, L, Dinv, af, muf, a, mu) && above_lambda_max(Af, Dinv, mu_f, mu, 1e-6);
        }
        if (!ok) {
            const Vec4d r = solve_f64_fallback(A[0][0], A[0][1], A[0][2], A[0][3], A[1][1], A[1][2], A[1][3],
                                               A[2][2], A[2][3], A[3][3], b[0], b[1], b[2], b[3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = r.v[k];
            return 1;
        }
        const double inv = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] *= inv;
        return 0;
    }
};

// Newton solve of the FP32 sweep.  The KKT system (mu - A) a = b, |a| = 1 is
// iterated from a = e0 (the current links) in the form
//   u = (mu - A)^-1 b,  y = (mu - A)^-1 a,
//   dmu = (a.u - 1 + s) / a.y  with s = (1 - a.a)/2,   a <- u - dmu y,
// which is the Newton step written without the residual b - (mu - A) a (the
// two solves share one LDL^T and run interleaved).  Stops when the correction
// is below 2e-6 or when the quadratic rate over the last two corrections puts
// the next one below it.  Returns true with a normalised when the accepted
// mu = mu_f + dmu (mu_f the multiplier of the last factorisation, dmu its
// step) is shown to lie above lambda_max(A), which makes a the global maximum
// (Sec. II.A): the pivots of mu_f - A are positive and above 1e-5 of the
// largest, and a step down (dmu < 0) stays below the smallest eigenvalue of
// mu_f - A with that margin.  The smallest eigenvalue is bounded from below
// by 27 det / tr^3 (det the product of the pivots, tr the trace; the other
// three eigenvalues have a product at most (tr / 3)^3).  Without the second
// test a step that crosses lambda_max near the hard case (beta_top ~ 0) would
// end on a stationary point that is not the maximum.  False otherwise.
__device__ __forceinline__ bool kkt_newton_f32(const float (&A)[4][4], const float (&b)[4], float (&a)[4]) {
    const float conv = 2e-6f;
    a[0] = 1.f;
    a[1] = a[2] = a[3] = 0.f;
    float mu = A[0][0] + b[0];
    float dprev = -1.f, dmin = 0.f, dabs = 0.f, dmu_last = 0.f;
    float D[4];
    bool ok = false;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        // LDL^T of M = mu - A
        float Dinv[4], L10, L20, L30, L21, L31, L32;
        D[0] = mu - A[0][0];
        Dinv[0] = frcp(D[0]);
        L10 = -A[1][0] * Dinv[0];
        L20 = -A[2][0] * Dinv[0];
        L30 = -A[3][0] * Dinv[0];
        D[1] = (mu - A[1][1]) - L10 * L10 * D[0];
        Dinv[1] = frcp(D[1]);
        L21 = (-A[2][1] - L20 * L10 * D[0]) * Dinv[1];
        L31 = (-A[3][1] - L30 * L10 * D[0]) * Dinv[1];
        D[2] = (mu - A[2][2]) - L20 * L20 * D[0] - L21 * L21 * D[1];
        Dinv[2] = frcp(D[2]);
        L32 = (-A[3][2] - L30 * L20 * D[0] - L31 * L21 * D[1]) * Dinv[2];
        D[3] = (mu - A[3][3]) - L30 * L30 * D[0] - L31 * L31 * D[1] - L32 * L32 * D[2];
        Dinv[3] = frcp(D[3]);
        dmin = fminf(fminf(D[0], D[1]), fminf(D[2], D[3]));
        dabs = fmaxf(fmaxf(fabsf(D[0]), fabsf(D[1])), fmaxf(fabsf(D[2]), fabsf(D[3])));
        const float dsmall = fminf(fminf(fabsf(D[0]), fabsf(D[1])), fminf(fabsf(D[2]), fabsf(D[3])));
        if (!(dsmall > 1e-12f * dabs)) return false;  // singular or NaN
        // u = M^-1 b, y = M^-1 a (forward, diagonal, backward substitution)
        float zu0 = b[0], zy0 = a[0];
        float zu1 = b[1] - L10 * zu0, zy1 = a[1] - L10 * zy0;
        float zu2 = b[2] - L20 * zu0 - L21 * zu1, zy2 = a[2] - L20 * zy0 - L21 * zy1;
        float zu3 = b[3] - L30 * zu0 - L31 * zu1 - L32 * zu2, zy3 = a[3] - L30 * zy0 - L31 * zy1 - L32 * zy2;
        zu0 *= Dinv[0]; zy0 *= Dinv[0];
        zu1 *= Dinv[1]; zy1 *= Dinv[1];
        zu2 *= Dinv[2]; zy2 *= Dinv[2];
        zu3 *= Dinv[3]; zy3 *= Dinv[3];
        const float u3 = zu3, y3 = zy3;
        const float u2 = zu2 - L32 * u3, y2 = zy2 - L32 * y3;
        const float u1 = zu1 - L21 * u2 - L31 * u3, y1 = zy1 - L21 * y2 - L31 * y3;
        const float u0 = zu0 - L10 * u1 - L20 * u2 - L30 * u3, y0 = zy0 - L10 * y1 - L20 * y2 - L30 * y3;
        const float aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
        const float au = a[0] * u0 + a[1] * u1 + a[2] * u2 + a[3] * u3;
        const float ay = a[0] * y0 + a[1] * y1 + a[2] * y2 + a[3] * y3;
        const float dmu = fdiv(au - 0.5f - 0.5f * aa, ay);
        const float n0 = u0 - dmu * y0, n1 = u1 - dmu * y1, n2 = u2 - dmu * y2, n3 = u3 - dmu * y3;
        const float dmax = fmaxf(fmaxf(fabsf(n0 - a[0]), fabsf(n1 - a[1])), fmaxf(fabsf(n2 - a[2]), fabsf(n3 - a[3])));
        a[0] = n0;
        a[1] = n1;
        a[2] = n2;
        a[3] = n3;
        mu += dmu;
        dmu_last = dmu;
        if (dmax <= conv || (dprev > 0.f && dmax * dmax * dmax <= conv * dprev * dprev)) {
            ok = true;
            break;
        }
        dprev = dmax;
    }
    if (!ok) return false;
    const float inv = rsqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] *= inv;
    if (!(dmin > 1e-5f * dabs)) return false;
    if (dmu_last < 0.f) {
        const float mf = mu - dmu_last;
        const float det = (D[0] * D[1]) * (D[2] * D[3]);
        const float tr = ((mf - A[0][0]) + (mf - A[1][1])) + ((mf - A[2][2]) + (mf - A[3][3]));
        return 27.f * det > (1e-5f * dabs - dmu_last) * (tr * tr * tr);
    }
    return true;
}

// FP32 fallback of the local solve (Jacobi + secular), out of line with its
// arguments and result passed by value so that the caller's A and b stay in
// registers.
static __device__ __noinline__ float4 solve_f32_fallback(float a00, float a01, float a02, float a03, float a11, float a12,
                                                  float a13, float a22, float a23, float a33, float b0, float b1,
                                                  float b2, float b3) {
    float S[4][4] = {{a00, a01, a02, a03}, {a01, a11, a12, a13}, {a02, a12, a22, a23}, {a03, a13, a23, a33}};
    const float b[4] = {b0, b1, b2, b3};
    float V[4][4], a[4], mu;
    jacobi4<float>(S, V, 8, 5e-7f);
    trs_from_eigen<float>(S, V, b, a, mu);
    // backstop: a degenerate local problem never feeds a non-finite update
    // into the links (the identity leaves the site unchanged)
    if (!(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]) && isfinite(a[3])))
        return make_float4(1.f, 0.f, 0.f, 0.f);
    return make_float4(a[0], a[1], a[2], a[3]);
}

// R partial sums: one per warp, partial[blockIdx.x * (NT / 32) + warp], summed
// by k_finalize in a fixed order (deterministic, and no block barrier in the
// sweep kernels).
__device__ __forceinline__ void warp_partial(double v, double* __restrict__ partial) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) partial[blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)] = v;
}

__device__ __forceinline__ int field_of_block(const FieldDesc* __restrict__ d, int nf, int b) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].blk0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
#ifdef MCG_CHECK
    mcg_bad(b < d[lo].blk0 || b >= d[lo].blk0 + d[lo].nblk);
#endif
    return lo;
}

}  // namespace mcg
