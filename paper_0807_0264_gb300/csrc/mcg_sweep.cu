// MCG relaxation on sm_103a: the checkerboard half-sweep kernel, the fused R
// reduction, per-field convergence control and the graph-captured sweep loop.
//
// Site update (Sec. II.A, MCG functional R = sum |tr U|^2; the update rule
// itself is the exact SU(2)-subgroup maximisation over subgroups (0,1),
// (0,2), (1,2)): for subgroup (p,q) the 8 links at x give
//   tr(G U_mu(x))        = c + w . a
//   tr(U_mu(x-mu) G^dag) = c + w' . a   (a_1..a_3 enter with a minus sign)
// for G the embedding of g = a0 + i a.sigma, so the local functional is
// a^T A a + 2 b.a + const with A = sum Re(conj(w) w^T), b = sum Re(conj(c) w),
// maximised on |a| = 1 (a trust-region subproblem: (mu - A) a = b with
// mu >= lambda_max(A)).
//
// Precision: the FP32 kernel does everything in FP32 (R accumulated in FP64).
// The FP64 kernel builds A, b and applies G in FP64; the 4x4 solve is seeded
// by an FP32 Jacobi eigen-decomposition + secular Newton and then refined to
// FP64 accuracy by Newton steps on the KKT system whose residual is evaluated
// in FP64 (the FP32 eigen-decomposition serves as the approximate inverse).
// Solves the refinement cannot settle (near-degenerate or hard cases) rerun
// in full FP64.  FP64 arithmetic is scarce on GB300, so the expensive part of
// the solve stays on the FP32 pipe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

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
    T beta[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) beta[i] = V[0][i] * b[0] + V[1][i] * b[1] + V[2][i] * b[2] + V[3][i] * b[3];
    T btop2 = T(0);
    bool top[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        top[i] = (amax - al[i]) <= deg_tol * scale;
        if (top[i]) btop2 += beta[i] * beta[i];
    }
    const T btop = fsqrt(btop2);
    if (btop <= hard_tol * scale) {
        T coef[4], pn2 = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            coef[i] = top[i] ? T(0) : fdiv(beta[i], amax - al[i]);
            pn2 += coef[i] * coef[i];
        }
        if (pn2 < T(1)) {
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
            T n2 = T(0);
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
    }
    // easy case: root of ||a(mu)|| = 1 right of amax, bracket [amax+btop, amax+||b||]
    T lo = amax + btop, hi = amax + bn, mu = lo;
    const int maxit = sizeof(T) == 8 ? 100 : 40;
#pragma unroll 1
    for (int it = 0; it < maxit; ++it) {
        T s2 = T(0), s3 = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // a zero weight contributes nothing (also when mu sits on al[i])
            if (beta[i] == T(0)) continue;
            const T r = frcp(mu - al[i]);
            const T q = beta[i] * beta[i] * r * r;
            s2 += q;
            s3 += q * r;
        }
        const T n = fsqrt(s2);
        if (n >= T(1))
            lo = fmax(lo, mu);
        else
            hi = fmin(hi, mu);
        T next = mu + fdiv((n - T(1)) * s2, s3);
        if (!(next > lo && next < hi)) next = T(0.5) * (lo + hi);
        if (fabs(next - mu) <= T(4) * eps * fabs(mu)) {
            mu = next;
            break;
        }
        mu = next;
        if (hi - lo <= T(4) * eps * fabs(mu)) break;
    }
    T n2 = T(0);
    T coef[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) coef[i] = beta[i] == T(0) ? T(0) : fdiv(beta[i], mu - al[i]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = V[k][0] * coef[0] + V[k][1] * coef[1] + V[k][2] * coef[2] + V[k][3] * coef[3];
        n2 += a[k] * a[k];
    }
    const T inv = rsqrt(n2);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] *= inv;
    mu_out = mu;
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
// success (converged, and mu - A positive definite: the global maximum of the
// trust-region subproblem) returns true with a normalised, mu, and the LDL^T
// factors of (mu - A) for later use.
template <typename T>
__device__ __forceinline__ bool kkt_newton(const T (&A)[4][4], const T (&b)[4], T (&a)[4], T& mu, T (&L)[4][4],
                                           T (&Dinv)[4], T& pd) {
    const T conv = sizeof(T) == 8 ? T(1e-13) : T(2e-6);
    a[0] = T(1);
    a[1] = a[2] = a[3] = T(0);
    mu = A[0][0] + b[0];
    bool ok = false;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
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
    // certificate: mu - A positive definite.  The factorization of the last
    // step (at mu - dmu, with |dmu| far below the pivot margin) serves.
    return pd > (sizeof(T) == 8 ? T(1e-12) : T(1e-5));
}

// FP32 solve of the subproblem given A (symmetric) and b (Jacobi + secular;
// out of line: the warm-started Newton path handles almost every solve).
__device__ __noinline__ int solve_f32(const float (&A)[4][4], const float (&b)[4], float (&a)[4], float& mu,
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
__device__ __noinline__ void solve_f64_full(const double* Ain, const double* b_in, double* a_out) {
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
                                                const float (&Dinv)[4], const float (&af)[4], float muf, double (&a)[4]) {
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
__device__ __noinline__ Vec4d solve_f64_fallback(double a00, double a01, double a02, double a03, double a11,
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
            float L[4][4], Dinv[4], pd;
            // warm-started FP32 Newton; the refinement contracts by ~cond * 1e-7,
            // with cond ~ 1 / pd bounded by the pivot test
            if (kkt_newton<float>(Af, bf, af, muf, L, Dinv, pd) && pd > 2e-4f)
                ok = kkt_refine_ldlt(A, b, L, Dinv, af, muf, a);
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
// the next one below it.  Returns true with a normalised when the last
// factorisation shows mu - A positive definite with pivots above 1e-5 of the
// largest (mu >= lambda_max: the global maximum), false otherwise.
__device__ __forceinline__ bool kkt_newton_f32(const float (&A)[4][4], const float (&b)[4], float (&a)[4]) {
    const float conv = 2e-6f;
    a[0] = 1.f;
    a[1] = a[2] = a[3] = 0.f;
    float mu = A[0][0] + b[0];
    float dprev = -1.f, dmin = 0.f, dabs = 0.f;
    bool ok = false;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        // LDL^T of M = mu - A
        float D[4], Dinv[4], L10, L20, L30, L21, L31, L32;
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
    // certificate from the last factorisation (at mu - dmu, |dmu| far below
    // the pivot margin)
    return dmin > 1e-5f * dabs;
}

// FP32 fallback of the local solve (Jacobi + secular), out of line with its
// arguments and result passed by value so that the caller's A and b stay in
// registers.
__device__ __noinline__ float4 solve_f32_fallback(float a00, float a01, float a02, float a03, float a11, float a12,
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

// ---------------------------------------------------------------------------
// link storage for one site's 8 links: shared memory, entry-major so that the
// threads of a warp touch consecutive addresses (conflict-free)
// ---------------------------------------------------------------------------
template <typename T, int NT>
struct SmemLinks {
    cplx<T>* base;
    __device__ __forceinline__ cplx<T>& operator()(int l, int e) { return base[(l * 9 + e) * NT + threadIdx.x]; }
};

// One SU(2)-subgroup step (subgroup rows/columns P, Q; R the third index) on
// the 8 links in shared memory (l < 4: forward U_l(x), 4 <= l < 8: backward
// U_{l-4}(x - l)) and Omega(x) (slot 8).  Returns 1 if the local solve left
// the fast path.
// S32 (FP64 links only): (A, b) are built and the local problem solved in
// FP32 (kkt_newton_f32, else the FP32 Jacobi path); the solution is
// normalised in FP64 so that G stays unitary to FP64 precision, and G is
// applied to the FP64 links as usual.
template <typename T, bool S32, typename L>
__device__ __forceinline__ int subgroup_step_s32(L& lk, const int P, const int Q, const int R, T (&a)[4]) {
    float A[4][4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        b[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) A[i][j] = 0.f;
    }
    const int ePP = 3 * P + P, ePQ = 3 * P + Q, eQP = 3 * Q + P, eQQ = 3 * Q + Q, eRR = 3 * R + R;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        const cplx<T> d11 = lk(l, ePP), d12 = lk(l, ePQ), d21 = lk(l, eQP), d22 = lk(l, eQQ), dc = lk(l, eRR);
        const cplx<float> m11 = mk((float)d11.x, (float)d11.y), m12 = mk((float)d12.x, (float)d12.y);
        const cplx<float> m21 = mk((float)d21.x, (float)d21.y), m22 = mk((float)d22.x, (float)d22.y);
        const cplx<float> c = mk((float)dc.x, (float)dc.y);
        cplx<float> w[4];
        w[0] = cadd(m11, m22);
        w[1] = mk(-(m21.y + m12.y), m21.x + m12.x);
        w[2] = csub(m21, m12);
        w[3] = mk(-(m11.y - m22.y), m11.x - m22.x);
        if (l >= 4) {
#pragma unroll
            for (int k = 1; k < 4; ++k) w[k] = mk(-w[k].x, -w[k].y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            b[k] = fmaf(c.x, w[k].x, fmaf(c.y, w[k].y, b[k]));
#pragma unroll
            for (int j = k; j < 4; ++j) A[k][j] = fmaf(w[k].x, w[j].x, fmaf(w[k].y, w[j].y, A[k][j]));
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < k; ++j) A[k][j] = A[j][k];
    float af[4];
    int fb = 0;
    if (!kkt_newton_f32(A, b, af)) {
        const float4 r = solve_f32_fallback(A[0][0], A[0][1], A[0][2], A[0][3], A[1][1], A[1][2], A[1][3], A[2][2],
                                            A[2][3], A[3][3], b[0], b[1], b[2], b[3]);
        af[0] = r.x;
        af[1] = r.y;
        af[2] = r.z;
        af[3] = r.w;
        fb = 1;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = (T)af[k];
    const T inv = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] *= inv;
    return fb;
}

// Coefficients of the local problem of subgroup (P, Q) at a site: the site's
// share of R after the move G(a) is a^T A a + 2 b^T a + const (Sec. II.A),
// with tr(G M) = M_RR + sum_k w_k a_k per link and w_1..w_3 negated for the
// backward links (which become M G^dag).
template <typename T, typename L>
__device__ __forceinline__ void local_problem(L& lk, const int P, const int Q, const int R, T (&A)[4][4],
                                              T (&b)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        b[i] = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) A[i][j] = T(0);
    }
    const int ePP = 3 * P + P, ePQ = 3 * P + Q, eQP = 3 * Q + P, eQQ = 3 * Q + Q, eRR = 3 * R + R;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        const cplx<T> m11 = lk(l, ePP), m12 = lk(l, ePQ), m21 = lk(l, eQP), m22 = lk(l, eQQ);
        const cplx<T> c = lk(l, eRR);
        cplx<T> w[4];
        w[0] = cadd(m11, m22);
        w[1] = mk(-(m21.y + m12.y), m21.x + m12.x);  // i (m21 + m12)
        w[2] = csub(m21, m12);
        w[3] = mk(-(m11.y - m22.y), m11.x - m22.x);  // i (m11 - m22)
        if (l >= 4) {
#pragma unroll
            for (int k = 1; k < 4; ++k) w[k] = mk(-w[k].x, -w[k].y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            b[k] = fma(c.x, w[k].x, fma(c.y, w[k].y, b[k]));
#pragma unroll
            for (int j = k; j < 4; ++j) A[k][j] = fma(w[k].x, w[j].x, fma(w[k].y, w[j].y, A[k][j]));
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < k; ++j) A[k][j] = A[j][k];
}

// The move itself: G = (a0 + i a3, a2 + i a1; -a2 + i a1, a0 - i a3) in rows
// and columns (P, Q); U_mu(x) <- G U_mu(x) and Omega(x) <- G Omega(x) (slots
// 0..3 and 8), U_mu(x - mu) <- U_mu(x - mu) G^dag (slots 4..7).
template <typename T, typename L>
__device__ __forceinline__ void apply_subgroup(L& lk, const int P, const int Q, const T (&a)[4]) {
    const cplx<T> g11 = mk(a[0], a[3]), g12 = mk(a[2], a[1]), g21 = mk(-a[2], a[1]), g22 = mk(a[0], -a[3]);
#pragma unroll 1
    for (int l = 0; l < 9; ++l) {
        if (l < 4 || l == 8) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {  // rows P, Q of G U (and of G Omega)
                const cplx<T> xp = lk(l, 3 * P + k), xq = lk(l, 3 * Q + k);
                lk(l, 3 * P + k) = cfma(g12, xq, cmul(g11, xp));
                lk(l, 3 * Q + k) = cfma(g22, xq, cmul(g21, xp));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {  // columns P, Q of U G^dag
                const cplx<T> xp = lk(l, 3 * k + P), xq = lk(l, 3 * k + Q);
                lk(l, 3 * k + P) = cfmac(xq, g12, cmulc(xp, g11));
                lk(l, 3 * k + Q) = cfmac(xq, g22, cmulc(xp, g21));
            }
        }
    }
}

template <typename T, typename L, bool S32 = false>
__device__ __forceinline__ int subgroup_step(L& lk, const int P, const int Q, const int R, const T omega) {
    T a[4];
    int fb;
    if constexpr (S32) {
        fb = subgroup_step_s32<T, S32>(lk, P, Q, R, a);
    } else {
        T A[4][4], b[4];
        local_problem<T>(lk, P, Q, R, A, b);
        asm volatile("" ::: "memory");
        fb = Solver<T>::solve(A, b, a);
    }
    if (omega != T(1)) {
        // over-relaxation: a -> normalise((1 - omega) e0 + omega a)
        a[0] = (T(1) - omega) + omega * a[0];
        a[1] *= omega;
        a[2] *= omega;
        a[3] *= omega;
        const T inv = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] *= inv;
    }
    apply_subgroup<T>(lk, P, Q, a);
    return fb;
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
    return lo;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Shared memory per thread: 8 links + Omega (81 complex): 41.5 KB for 64 FP32
// threads (5 blocks per SM), 83 KB for 128 FP32 or 64 FP64 threads (2 per SM).
template <typename T, bool ACC, int NT, bool S32 = false>
__global__ void __launch_bounds__(NT, 2) k_halfsweep(SweepBatch bt, int parity) {
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    if (bt.state[f].done) return;  // block-uniform
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    cplx<T>* __restrict__ U = reinterpret_cast<cplx<T>*>(fd.U);
    cplx<T>* __restrict__ G = reinterpret_cast<cplx<T>*>(fd.G);
    const int s = (blockIdx.x - fd.blk0) * NT + threadIdx.x;
    const bool active = s < g.vh;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemLinks<T, NT> lk;
    lk.base = reinterpret_cast<cplx<T>*>(smem_raw);

    double rsum = 0.0;
    int fb = 0;
    if (active) {
        int c[4];
        eo_coords(g, parity, s, c);
        int sb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) sb[mu] = eo_neighbor(g, c, mu, -1);
        // stage the 8 links and Omega in shared memory without passing
        // through registers
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const cplx<T>* src = U + lidx(g, mu, parity, 0, s);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<T>)>(&lk(mu, e), src + (size_t)e * g.vh);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const cplx<T>* src = U + lidx(g, mu, parity ^ 1, 0, sb[mu]);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<T>)>(&lk(4 + mu, e), src + (size_t)e * g.vh);
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<T>)>(&lk(8, e), &G[gidx(g, parity, e, s)]);
        cp_async_wait_all();

        // subgroups (0,1), (0,2), (1,2) in turn; compiler barriers keep the
        // links in shared memory between the phases of the update
        const T omega = (T)bt.omega;
#pragma unroll 1
        for (int sg = 0; sg < 3; ++sg) {
            const int P = sg == 2 ? 1 : 0, Q = sg == 0 ? 1 : 2;
            fb += subgroup_step<T, SmemLinks<T, NT>, S32>(lk, P, Q, 3 - P - Q, omega);
            asm volatile("" ::: "memory");
        }

#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cplx<T>* dst = U + lidx(g, mu, parity, 0, s);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) dst[(size_t)e * g.vh] = lk(mu, e);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cplx<T>* dst = U + lidx(g, mu, parity ^ 1, 0, sb[mu]);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) dst[(size_t)e * g.vh] = lk(4 + mu, e);
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) G[gidx(g, parity, e, s)] = lk(8, e);
        if (ACC) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const T tr = lk(l, 0).x + lk(l, 4).x + lk(l, 8).x;
                const T ti = lk(l, 0).y + lk(l, 4).y + lk(l, 8).y;
                rsum += (double)tr * (double)tr + (double)ti * (double)ti;
            }
        }
    }
    if (ACC) warp_partial(rsum, bt.partial);
    {
        // count local solves that left the fast path (diagnostic)
        const int w = __reduce_add_sync(0xffffffffu, fb);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&bt.state[f].fallbacks, w);
    }
}

// ---------------------------------------------------------------------------
// Simulated annealing of the gauge transform (Sec. III.B names annealing as the
// SU(2) route to higher maxima; here a Gribov-copy search variant run ahead
// of the relaxation).  Each subgroup of a site gets nhit Metropolis hits on
// the same move as the relaxation; the local problem (A, b) is built once per
// subgroup, the hits are composed as SU(2) elements relative to it and scored
// by the quadratic form, and the accepted product is applied once.
// ---------------------------------------------------------------------------

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)), the key advancing by the Weyl increments between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long (&c)[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        c[0] = hi1 ^ c[1] ^ k0;
        c[1] = lo1;
        c[2] = hi0 ^ c[3] ^ k1;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// top 53 bits -> [0, 1), exact
__device__ __forceinline__ double unit_interval(unsigned long long w) { return (double)(w >> 11) * 0x1p-53; }

// a^T A a + 2 b^T a
__device__ __forceinline__ double local_quadratic(const double (&A)[4][4], const double (&b)[4], const double (&a)[4]) {
    double f = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double r = 2.0 * b[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) r = fma(A[i][j], a[j], r);
        f = fma(r, a[i], f);
    }
    return f;
}

struct AnnealArgs {
    cplx<double>* U;
    cplx<double>* G;
    Geom g;
    double T;
    long long sweep;
    int nhit;
    double eps;
    unsigned long long seed;
    unsigned long long* accepted;  // one per field
};

// One annealing half-sweep over the sites of `parity`, one thread per site,
// field blockIdx.y.  The random words of hit h of subgroup s at
// lexicographic site x come from the counter (x, sweep, s * nhit + h, field)
// under key (seed, 0): v_k = eps (2 u_k - 1), a0 = sqrt(1 - |v|^2) (rounded
// step by step, no contraction), accepted when dF >= 0 or u_3 < exp(dF / T).
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_anneal_halfsweep(AnnealArgs an, int parity) {
    const int f = blockIdx.y;
    const Geom g = an.g;
    cplx<double>* __restrict__ U = an.U + (size_t)f * link_elems(g);
    cplx<double>* __restrict__ G = an.G + (size_t)f * gauge_elems(g);
    const int s = blockIdx.x * NT + threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemLinks<double, NT> lk;
    lk.base = reinterpret_cast<cplx<double>*>(smem_raw);

    unsigned int acc = 0;
    if (s < g.vh) {
        int c[4];
        eo_coords(g, parity, s, c);
        int sb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) sb[mu] = eo_neighbor(g, c, mu, -1);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const cplx<double>* src = U + lidx(g, mu, parity, 0, s);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<double>)>(&lk(mu, e), src + (size_t)e * g.vh);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const cplx<double>* src = U + lidx(g, mu, parity ^ 1, 0, sb[mu]);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<double>)>(&lk(4 + mu, e), src + (size_t)e * g.vh);
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) cp_async<sizeof(cplx<double>)>(&lk(8, e), &G[gidx(g, parity, e, s)]);
        cp_async_wait_all();

        const unsigned long long x =
            (unsigned long long)c[0] +
            (unsigned long long)g.n[0] * (c[1] + (unsigned long long)g.n[1] * (c[2] + (unsigned long long)g.n[2] * c[3]));
        const double T = an.T, eps = an.eps;
#pragma unroll 1
        for (int sg = 0; sg < 3; ++sg) {
            const int P = sg == 2 ? 1 : 0, Q = sg == 0 ? 1 : 2;
            double A[4][4], b[4];
            local_problem<double>(lk, P, Q, 3 - P - Q, A, b);
            double cur[4] = {1.0, 0.0, 0.0, 0.0};
            double Fcur = local_quadratic(A, b, cur);
#pragma unroll 1
            for (int h = 0; h < an.nhit; ++h) {
                unsigned long long w[4] = {x, (unsigned long long)an.sweep, (unsigned long long)(sg * an.nhit + h),
                                           (unsigned long long)f};
                philox4x64_10(w, an.seed, 0ull);
                const double v1 = __dmul_rn(eps, __dsub_rn(__dmul_rn(2.0, unit_interval(w[0])), 1.0));
                const double v2 = __dmul_rn(eps, __dsub_rn(__dmul_rn(2.0, unit_interval(w[1])), 1.0));
                const double v3 = __dmul_rn(eps, __dsub_rn(__dmul_rn(2.0, unit_interval(w[2])), 1.0));
                const double a0 =
                    __dsqrt_rn(__dsub_rn(1.0, __dadd_rn(__dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2)), __dmul_rn(v3, v3))));
                // candidate = proposal * current (SU(2) product in (a0, a) form)
                double cand[4];
                cand[0] = a0 * cur[0] - (v1 * cur[1] + v2 * cur[2] + v3 * cur[3]);
                cand[1] = a0 * cur[1] + cur[0] * v1 - (v2 * cur[3] - v3 * cur[2]);
                cand[2] = a0 * cur[2] + cur[0] * v2 - (v3 * cur[1] - v1 * cur[3]);
                cand[3] = a0 * cur[3] + cur[0] * v3 - (v1 * cur[2] - v2 * cur[1]);
                const double Fc = local_quadratic(A, b, cand);
                const double dF = Fc - Fcur;
                if (dF >= 0.0 || unit_interval(w[3]) < exp(dF / T)) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) cur[k] = cand[k];
                    Fcur = Fc;
                    ++acc;
                }
            }
            const double inv = rsqrt(cur[0] * cur[0] + cur[1] * cur[1] + cur[2] * cur[2] + cur[3] * cur[3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) cur[k] *= inv;
            apply_subgroup<double>(lk, P, Q, cur);
            asm volatile("" ::: "memory");
        }

#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cplx<double>* dst = U + lidx(g, mu, parity, 0, s);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) dst[(size_t)e * g.vh] = lk(mu, e);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cplx<double>* dst = U + lidx(g, mu, parity ^ 1, 0, sb[mu]);
#pragma unroll 1
            for (int e = 0; e < 9; ++e) dst[(size_t)e * g.vh] = lk(4 + mu, e);
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) G[gidx(g, parity, e, s)] = lk(8, e);
    }
    const unsigned int w = __reduce_add_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&an.accepted[f], (unsigned long long)w);
}

// ---------------------------------------------------------------------------
// FP32 half-sweep on the compact storage: one thread per site, the site's
// nine matrices (forward links U_mu(x), backward links U_mu(x - mu), W(x)) in
// registers as their rows 0 and 1 (108 floats), the three subgroup steps
// unrolled with compile-time indices.  Row-2 entries are rebuilt where a step
// needs them; G acting on rows (P, 2) of a forward link changes row P only in
// the stored part (row 2 stays implied), and M G^dag acts on each row of a
// backward link separately.  No shared memory: the loads of all nine matrices
// are in flight at once, straight into registers.
// ---------------------------------------------------------------------------

// Makes the compiler treat the forward links as redefined here (no code
// emitted): values derived from them before this point (row-2 entries built
// for A and b) are recomputed after it instead of being held in registers
// across the local solve.
__device__ __forceinline__ void c12_opaque(cplx<float> (&m)[4][6]) {
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int e = 0; e < 6; ++e) asm volatile("" : "+f"(m[l][e].x), "+f"(m[l][e].y));
}

template <int I, int J>
__device__ __forceinline__ cplx<float> c12_entry(const cplx<float>* m) {
    if constexpr (I < 2)
        return m[3 * I + J];
    else
        return row2_entry(m, J);
}

// M <- G M for the subgroup element G = a0 + i a.sigma embedded at rows and
// columns (P, Q), on a compact matrix (rows 0 and 1).  For Q = 2 only row P
// of the stored part changes; the new row 2 stays implied.
template <int P, int Q>
__device__ __forceinline__ void c12_left_update(cplx<float>* m, const float (&a)[4]) {
    const cplx<float> g11 = mk(a[0], a[3]), g12 = mk(a[2], a[1]), g21 = mk(-a[2], a[1]), g22 = mk(a[0], -a[3]);
    if constexpr (Q < 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cplx<float> xp = m[3 * P + k], xq = m[3 * Q + k];
            m[3 * P + k] = cfma(g12, xq, cmul(g11, xp));
            m[3 * Q + k] = cfma(g22, xq, cmul(g21, xp));
        }
    } else {
        cplx<float> r2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r2[k] = row2_entry(m, k);
#pragma unroll
        for (int k = 0; k < 3; ++k) m[3 * P + k] = cfma(g12, r2[k], cmul(g11, m[3 * P + k]));
    }
}

// Backward links U_mu(x - mu) of the site live in shared memory as compact
// chunks, slot (l, q) of thread t at bst[(l*3 + q)*NT + t] (consecutive
// threads, consecutive 16-byte words).
template <int NT>
__device__ __forceinline__ void bwd_load(const float4* bst, int l, cplx<float>* m) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 v = bst[(l * 3 + q) * NT + threadIdx.x];
        m[2 * q] = mk(v.x, v.y);
        m[2 * q + 1] = mk(v.z, v.w);
    }
}
template <int NT>
__device__ __forceinline__ void bwd_store(float4* bst, int l, const cplx<float>* m) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
        bst[(l * 3 + q) * NT + threadIdx.x] = make_float4(m[2 * q].x, m[2 * q].y, m[2 * q + 1].x, m[2 * q + 1].y);
}

// Packed FP32 arithmetic: on sm_100 and later one instruction performs two
// independent FP32 FMAs on a register pair (__ffma2_rn), which halves the
// instruction count of the (A, b) build and of the SU(2) moves.  A complex
// number is such a pair.  The moves use g x = g.x (x.x, x.y) + g.y (-x.y, x.x),
// with the coefficients of the subgroup element broadcast to pairs once per
// step: x[i] = (g_i.x, g_i.x), y[i] = (-g_i.y, g_i.y), yc[i] = (g_i.y, -g_i.y)
// for g_i = g11, g12, g21, g22.
struct PackedSU2 {
    float2 x[4], y[4], yc[4];
};
__device__ __forceinline__ void packed_su2(const float (&a)[4], PackedSU2& G) {
    const float gx[4] = {a[0], a[2], -a[2], a[0]};
    const float gy[4] = {a[3], a[1], a[1], -a[3]};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        G.x[i] = make_float2(gx[i], gx[i]);
        G.y[i] = make_float2(-gy[i], gy[i]);
        G.yc[i] = make_float2(gy[i], -gy[i]);
    }
}
__device__ __forceinline__ float2 pk(cplx<float> c) { return make_float2(c.x, c.y); }
__device__ __forceinline__ float2 pk_swap(cplx<float> c) { return make_float2(c.y, c.x); }
// g_i0 u + g_i1 v  (a row of G M)
__device__ __forceinline__ cplx<float> su2_row(const PackedSU2& G, int i0, int i1, cplx<float> u, cplx<float> v) {
    float2 r = __fmul2_rn(G.x[i0], pk(u));
    r = __ffma2_rn(G.y[i0], pk_swap(u), r);
    r = __ffma2_rn(G.x[i1], pk(v), r);
    r = __ffma2_rn(G.y[i1], pk_swap(v), r);
    return mk(r.x, r.y);
}
// u conj(g_i0) + v conj(g_i1)  (an entry of M G^dag)
__device__ __forceinline__ cplx<float> su2_col(const PackedSU2& G, int i0, int i1, cplx<float> u, cplx<float> v) {
    float2 r = __fmul2_rn(G.x[i0], pk(u));
    r = __ffma2_rn(G.yc[i0], pk_swap(u), r);
    r = __ffma2_rn(G.x[i1], pk(v), r);
    r = __ffma2_rn(G.yc[i1], pk_swap(v), r);
    return mk(r.x, r.y);
}
// M <- G M on a compact matrix (rows 0 and 1), as c12_left_update.
template <int P, int Q>
__device__ __forceinline__ void c12_left_update_pk(cplx<float>* m, const PackedSU2& G) {
    if constexpr (Q < 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const cplx<float> xp = m[3 * P + k], xq = m[3 * Q + k];
            m[3 * P + k] = su2_row(G, 0, 1, xp, xq);
            m[3 * Q + k] = su2_row(G, 2, 3, xp, xq);
        }
    } else {
        cplx<float> r2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r2[k] = row2_entry(m, k);
#pragma unroll
        for (int k = 0; k < 3; ++k) m[3 * P + k] = su2_row(G, 0, 1, m[3 * P + k], r2[k]);
    }
}

// One SU(2)-subgroup step (rows/columns P < Q, R the third index) on the
// compact forward links m[0..3] (registers) and the compact backward links
// in shared memory.  Writes the (over-relaxed) subgroup element to `a` for the
// update of W; returns 1 if the local solve left the Newton path.
template <int P, int Q, int R, int NT>
__device__ __forceinline__ int c12_subgroup_step(cplx<float> (&m)[4][6], float4* bst, const float omega,
                                                 float (&a)[4]) {
    // A = sum Re(conj(w) w^T), b = sum Re(conj(c) w): each entry accumulated as
    // a pair (sum of x-products, sum of y-products), added at the end.  For a
    // backward link w_1..w_3 change sign, which flips b_1..b_3 and A_0j (j > 0).
    float2 Ap[10], bp[4];
#pragma unroll
    for (int i = 0; i < 10; ++i) Ap[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) bp[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        cplx<float> mb[6];
        if (l >= 4) bwd_load<NT>(bst, l - 4, mb);
        const cplx<float>* M = l < 4 ? m[l] : mb;
        const cplx<float> m11 = c12_entry<P, P>(M), m12 = c12_entry<P, Q>(M);
        const cplx<float> m21 = c12_entry<Q, P>(M), m22 = c12_entry<Q, Q>(M);
        const cplx<float> cc = c12_entry<R, R>(M);
        // tr(G M) = cc + w.a, w = (m11 + m22, i(m21 + m12), m21 - m12, i(m11 - m22))
        float2 w[4];
        w[0] = make_float2(m11.x + m22.x, m11.y + m22.y);
        w[1] = make_float2(-(m21.y + m12.y), m21.x + m12.x);
        w[2] = make_float2(m21.x - m12.x, m21.y - m12.y);
        w[3] = make_float2(-(m11.y - m22.y), m11.x - m22.x);
        float2 c0 = make_float2(cc.x, cc.y), c1 = c0, w0 = w[0];
        if (l >= 4) {
            c1 = make_float2(-cc.x, -cc.y);
            w0 = make_float2(-w[0].x, -w[0].y);
        }
        bp[0] = __ffma2_rn(c0, w[0], bp[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k) bp[k] = __ffma2_rn(c1, w[k], bp[k]);
        Ap[0] = __ffma2_rn(w[0], w[0], Ap[0]);
        Ap[1] = __ffma2_rn(w0, w[1], Ap[1]);
        Ap[2] = __ffma2_rn(w0, w[2], Ap[2]);
        Ap[3] = __ffma2_rn(w0, w[3], Ap[3]);
        Ap[4] = __ffma2_rn(w[1], w[1], Ap[4]);
        Ap[5] = __ffma2_rn(w[1], w[2], Ap[5]);
        Ap[6] = __ffma2_rn(w[1], w[3], Ap[6]);
        Ap[7] = __ffma2_rn(w[2], w[2], Ap[7]);
        Ap[8] = __ffma2_rn(w[2], w[3], Ap[8]);
        Ap[9] = __ffma2_rn(w[3], w[3], Ap[9]);
    }
    float A[4][4], b[4];
    {
        int i = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = k; j < 4; ++j, ++i) A[k][j] = A[j][k] = Ap[i].x + Ap[i].y;
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = bp[k].x + bp[k].y;
    }
    c12_opaque(m);
    asm volatile("" ::: "memory");
    int fb = 0;
    if (!kkt_newton_f32(A, b, a)) {
        const float4 r = solve_f32_fallback(A[0][0], A[0][1], A[0][2], A[0][3], A[1][1], A[1][2], A[1][3], A[2][2],
                                            A[2][3], A[3][3], b[0], b[1], b[2], b[3]);
        a[0] = r.x;
        a[1] = r.y;
        a[2] = r.z;
        a[3] = r.w;
        fb = 1;
    }
    if (omega != 1.f) {
        // over-relaxation: a -> normalise((1 - omega) e0 + omega a)
        a[0] = (1.f - omega) + omega * a[0];
        a[1] *= omega;
        a[2] *= omega;
        a[3] *= omega;
        const float inv = rsqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] *= inv;
    }
    PackedSU2 G;
    packed_su2(a, G);
    // forward links: rows P, Q of G M
#pragma unroll
    for (int l = 0; l < 4; ++l) c12_left_update_pk<P, Q>(m[l], G);
    // backward links: columns P, Q of M G^dag, rows 0 and 1
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        cplx<float> mb[6];
        bwd_load<NT>(bst, l, mb);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const cplx<float> xp = mb[3 * i + P], xq = mb[3 * i + Q];
            mb[3 * i + P] = su2_col(G, 0, 1, xp, xq);
            mb[3 * i + Q] = su2_col(G, 2, 3, xp, xq);
        }
        bwd_store<NT>(bst, l, mb);
    }
    asm volatile("" ::: "memory");
    return fb;
}

// One thread per site.  The 4 forward links are loaded straight into
// registers (12 16-byte loads in flight); the 4 backward links and W are
// staged into shared memory by cp.async meanwhile.  The backward links are
// read and written there by each subgroup step; W, needed only after the
// three steps, is updated at the end with the three subgroup elements.
// Keeping half of the site's state out of registers removes most spills at
// the 168-register budget of 3 blocks of 128 threads per SM.
template <bool ACC, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_halfsweep_c12(SweepBatch bt, int parity) {
    extern __shared__ float4 c12_smem[];  // W: 3 chunks x NT, then backward links: 12 chunks x NT
    float4* wstage = c12_smem;
    float4* bst = c12_smem + 3 * NT;
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    if (bt.state[f].done) return;  // block-uniform
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    float4* __restrict__ U = reinterpret_cast<float4*>(fd.U);
    float4* __restrict__ W = reinterpret_cast<float4*>(fd.G);
    const int s = (blockIdx.x - fd.blk0) * NT + threadIdx.x;
    const size_t vh = (size_t)g.vh;
    float rsum = 0.f;
    int fb = 0;
    if (s < g.vh) {
        int c[4];
        eo_coords(g, parity, s, c);
        int sb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) sb[mu] = eo_neighbor(g, c, mu, -1);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const float4* src = U + c12_lidx(g, mu, parity ^ 1, 0, sb[mu]);
#pragma unroll
            for (int q = 0; q < 3; ++q) cp_async<16>(&bst[(mu * 3 + q) * NT + threadIdx.x], src + q * vh);
        }
        {
            const float4* src = W + c12_gidx(g, parity, 0, s);
#pragma unroll
            for (int q = 0; q < 3; ++q) cp_async<16>(&wstage[q * NT + threadIdx.x], src + q * vh);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        cplx<float> m[4][6];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) c12_load(U + c12_lidx(g, mu, parity, 0, s), vh, m[mu]);
        cp_async_wait_all();

        const float omega = (float)bt.omega;
        float a01[4], a02[4], a12[4];
        fb += c12_subgroup_step<0, 1, 2, NT>(m, bst, omega, a01);
        fb += c12_subgroup_step<0, 2, 1, NT>(m, bst, omega, a02);
        fb += c12_subgroup_step<1, 2, 0, NT>(m, bst, omega, a12);

        // FP32 re-unitarisation every sweep: the 8 links in the odd half-sweep
        // (which touches every link once), W every half-sweep.  FP32 rounding
        // would otherwise inflate |tr U|^2 by ~1e-6 per sweep and swamp the
        // convergence signal.  R: the site's 8 links (|tr|^2 <= 9 each) summed
        // in FP32, widened once.
        if (ACC) {
#pragma unroll
            for (int l = 0; l < 4; ++l) c12_reunitarise(m[l]);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) c12_store(U + c12_lidx(g, mu, parity, 0, s), vh, m[mu]);
        if (ACC) {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const cplx<float> t = cadd(cadd(m[l][0], m[l][4]), row2_entry(m[l], 2));
                rsum = fmaf(t.x, t.x, fmaf(t.y, t.y, rsum));
            }
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cplx<float> mb[6];
            bwd_load<NT>(bst, mu, mb);
            if (ACC) {
                c12_reunitarise(mb);
                const cplx<float> t = cadd(cadd(mb[0], mb[4]), row2_entry(mb, 2));
                rsum = fmaf(t.x, t.x, fmaf(t.y, t.y, rsum));
            }
            c12_store(U + c12_lidx(g, mu, parity ^ 1, 0, sb[mu]), vh, mb);
        }
        cplx<float> w[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 v = wstage[q * NT + threadIdx.x];
            w[2 * q] = mk(v.x, v.y);
            w[2 * q + 1] = mk(v.z, v.w);
        }
        PackedSU2 G;
        packed_su2(a01, G);
        c12_left_update_pk<0, 1>(w, G);
        packed_su2(a02, G);
        c12_left_update_pk<0, 2>(w, G);
        packed_su2(a12, G);
        c12_left_update_pk<1, 2>(w, G);
        c12_reunitarise(w);
        c12_store(W + c12_gidx(g, parity, 0, s), vh, w);
    }
    if (ACC) warp_partial((double)rsum, bt.partial);
    {
        // count local solves that left the Newton path (diagnostic)
        const int w = __reduce_add_sync(0xffffffffu, fb);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&bt.state[f].fallbacks, w);
    }
}

// R over all links of each field, into per-block partials (same block map as
// the half-sweep).  FP64 fields are in the full layout, FP32 fields in the
// compact one (tr U = U00 + U11 + conj(U00 U11 - U01 U10)).
template <typename T>
__global__ void __launch_bounds__(256) k_functional(SweepBatch bt) {
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    const int s = (blockIdx.x - fd.blk0) * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (s < g.vh) {
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                double tr, ti;
                if constexpr (sizeof(T) == 8) {
                    const cplx<T>* __restrict__ U = reinterpret_cast<const cplx<T>*>(fd.U);
                    const cplx<T> a = U[lidx(g, mu, p, 0, s)], b = U[lidx(g, mu, p, 4, s)], c = U[lidx(g, mu, p, 8, s)];
                    tr = (double)(a.x + b.x + c.x);
                    ti = (double)(a.y + b.y + c.y);
                } else {
                    const float4* __restrict__ U = reinterpret_cast<const float4*>(fd.U);
                    cplx<float> m[6];
                    c12_load(U + c12_lidx(g, mu, p, 0, s), (size_t)g.vh, m);
                    const cplx<float> t = cadd(cadd(m[0], m[4]), row2_entry(m, 2));
                    tr = (double)t.x;
                    ti = (double)t.y;
                }
                r += tr * tr + ti * ti;
            }
    }
    warp_partial(r, bt.partial);
}

// mode 0: end of a sweep; 1: fresh start (sweep = 0); 2: continue (new phase)
__global__ void __launch_bounds__(256) k_finalize(SweepBatch bt, int mode) {
    const int f = blockIdx.x;
    FieldState* st = &bt.state[f];
    if (mode == 0 && st->done) {
        if (threadIdx.x == 0) st->reunit_pending = 0;
        return;
    }
    const FieldDesc fd = bt.desc[f];
    double v = 0.0;
    const size_t n = (size_t)fd.nblk * bt.ppb;
    const double* __restrict__ part = bt.partial + (size_t)fd.blk0 * bt.ppb;
    for (size_t k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
    __shared__ double red[8];
    const double R = block_sum(v, red);
    if (threadIdx.x != 0) return;
    if (mode != 0) {
        if (mode == 1) {
            st->sweep = 0;
            st->fallbacks = 0;
            if (bt.R_hist) bt.R_hist[(size_t)f * bt.hist_len] = R;
        }
        st->R_prev = R;
        st->R_last = R;
        st->reunit_pending = 0;
        st->phase_start = st->sweep;
        st->ring[st->sweep % kRing] = R;
        st->done = st->sweep >= st->max_sweeps ? 2 : 0;
        return;
    }
    const int k = st->sweep + 1;
    st->sweep = k;
    if (bt.R_hist && k < bt.hist_len) bt.R_hist[(size_t)f * bt.hist_len + k] = R;
    // dV per sweep, averaged over the last `window` sweeps of this phase
    double dV;
    if (bt.window <= 1) {
        dV = (R - st->R_prev) * fd.norm;
    } else if (k - st->phase_start >= bt.window) {
        dV = (R - st->ring[(k - bt.window) % kRing]) * fd.norm / bt.window;
    } else {
        dV = 1e300;
    }
    st->ring[k % kRing] = R;
    st->R_prev = R;
    st->R_last = R;
    st->reunit_pending = (bt.reunit_every > 0 && k % bt.reunit_every == 0) ? 1 : 0;
    if (dV < bt.tol)
        st->done = 1;
    else if (k >= st->max_sweeps)
        st->done = 2;
}

// Re-unitarise the links and Omega of fields with reunit_pending set.
template <typename T>
__global__ void __launch_bounds__(128) k_reunit_pending(SweepBatch bt) {
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    if (!bt.state[f].reunit_pending) return;
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    cplx<T>* __restrict__ U = reinterpret_cast<cplx<T>*>(fd.U);
    cplx<T>* __restrict__ G = reinterpret_cast<cplx<T>*>(fd.G);
    const int s = (blockIdx.x - fd.blk0) * blockDim.x + threadIdx.x;
    if (s >= g.vh) return;
    for (int p = 0; p < 2; ++p) {
        cplx<T> m[9];
        for (int mu = 0; mu < 4; ++mu) {
            load_link(U, g, mu, p, s, m);
            m3_reunitarise(m);
            store_link(U, g, mu, p, s, m);
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = G[gidx(g, p, e, s)];
        m3_reunitarise(m);
#pragma unroll
        for (int e = 0; e < 9; ++e) G[gidx(g, p, e, s)] = m[e];
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
// Threads per block of the half-sweep kernel, per precision; set by
// mcg_set_sweep_block (the block-size autotuner).  Both run one thread per
// site: FP64 64 or 128 threads, FP32 (compact, register resident) 64, 128 or
// 256.
static int g_sweep_nt[2] = {128, 128};

int sweep_block(int prec) { return g_sweep_nt[prec == MCG_F64 ? 0 : 1]; }
void set_sweep_block(int prec, int nt) { g_sweep_nt[prec == MCG_F64 ? 0 : 1] = nt; }
int sweep_sites_per_block(int prec) { return sweep_block(prec); }

template <typename K>
static int raise_smem(K kernel, size_t smem) {
    MCG_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return 0;
}

// shared memory of the FP64 kernel: 8 links + Omega per thread
static size_t halfsweep_smem_f64(int nt) { return sizeof(cplx<double>) * 81 * nt; }

// FP32 kernel: dynamic shared memory for the staged W and backward links
// (15 chunks per thread: 30 KB for 128 threads)
static size_t halfsweep_smem_c12(int nt) { return sizeof(float4) * 15 * nt; }

// Raises the dynamic shared-memory limit of the half-sweep kernels for the
// current device.  Called on every fix phase (never inside a stream capture):
// the attribute is per device, and the call costs microseconds.
template <typename T>
static int prepare_halfsweep(int nt) {
    if constexpr (sizeof(T) == 8) {
        const size_t smem = halfsweep_smem_f64(nt);
        int rc = 0;
        if (nt == 128) {
            if ((rc = raise_smem(k_halfsweep<T, false, 128>, smem)) || (rc = raise_smem(k_halfsweep<T, true, 128>, smem)) ||
                (rc = raise_smem(k_halfsweep<T, false, 128, true>, smem)) ||
                (rc = raise_smem(k_halfsweep<T, true, 128, true>, smem)))
                return rc;
        } else {
            if ((rc = raise_smem(k_halfsweep<T, false, 64>, smem)) || (rc = raise_smem(k_halfsweep<T, true, 64>, smem)) ||
                (rc = raise_smem(k_halfsweep<T, false, 64, true>, smem)) ||
                (rc = raise_smem(k_halfsweep<T, true, 64, true>, smem)))
                return rc;
        }
    } else {
        const size_t smem = halfsweep_smem_c12(nt);
        int rc = 0;
        if (nt == 256) {
            if ((rc = raise_smem(k_halfsweep_c12<false, 256, 1>, smem)) ||
                (rc = raise_smem(k_halfsweep_c12<true, 256, 1>, smem)))
                return rc;
        } else if (nt == 128) {
            if ((rc = raise_smem(k_halfsweep_c12<false, 128, 3>, smem)) ||
                (rc = raise_smem(k_halfsweep_c12<true, 128, 3>, smem)))
                return rc;
        } else {
            if ((rc = raise_smem(k_halfsweep_c12<false, 64, 6>, smem)) ||
                (rc = raise_smem(k_halfsweep_c12<true, 64, 6>, smem)))
                return rc;
        }
    }
    return 0;
}

// FP32 occupancy: the register file holds 3 blocks of 128 threads (<= 168
// registers per thread).
template <typename T>
static void launch_halfsweep(int nt, bool acc, const SweepBatch& bt, int parity, int nblocks, cudaStream_t st) {
    if constexpr (sizeof(T) == 8) {
        const size_t smem = halfsweep_smem_f64(nt);
        const bool s32 = bt.solve32 != 0;
        if (nt == 128) {
            if (acc)
                (s32 ? k_halfsweep<T, true, 128, true> : k_halfsweep<T, true, 128>)<<<nblocks, 128, smem, st>>>(bt, parity);
            else
                (s32 ? k_halfsweep<T, false, 128, true> : k_halfsweep<T, false, 128>)<<<nblocks, 128, smem, st>>>(bt,
                                                                                                                parity);
        } else {
            if (acc)
                (s32 ? k_halfsweep<T, true, 64, true> : k_halfsweep<T, true, 64>)<<<nblocks, 64, smem, st>>>(bt, parity);
            else
                (s32 ? k_halfsweep<T, false, 64, true> : k_halfsweep<T, false, 64>)<<<nblocks, 64, smem, st>>>(bt, parity);
        }
    } else {
        const size_t smem = halfsweep_smem_c12(nt);
        const int grid = nblocks;
        if (nt == 256) {
            if (acc)
                k_halfsweep_c12<true, 256, 1><<<grid, 256, smem, st>>>(bt, parity);
            else
                k_halfsweep_c12<false, 256, 1><<<grid, 256, smem, st>>>(bt, parity);
        } else if (nt == 128) {
            if (acc)
                k_halfsweep_c12<true, 128, 3><<<grid, 128, smem, st>>>(bt, parity);
            else
                k_halfsweep_c12<false, 128, 3><<<grid, 128, smem, st>>>(bt, parity);
        } else {
            if (acc)
                k_halfsweep_c12<true, 64, 6><<<grid, 64, smem, st>>>(bt, parity);
            else
                k_halfsweep_c12<false, 64, 6><<<grid, 64, smem, st>>>(bt, parity);
        }
    }
}

template <typename T>
static int enqueue_sweep(const SweepBatch& bt, int nt, int spb, cudaStream_t st) {
    launch_halfsweep<T>(nt, false, bt, 0, bt.total_blocks, st);
    launch_halfsweep<T>(nt, true, bt, 1, bt.total_blocks, st);
    k_finalize<<<bt.nf, 256, 0, st>>>(bt, 0);
    // FP32 sweeps re-unitarise inside the half-sweep kernel
    if constexpr (sizeof(T) == 8)
        if (bt.reunit_every > 0) k_reunit_pending<T><<<bt.total_blocks, spb, 0, st>>>(bt);
    return 0;
}

template <typename T>
int run_fix_phase(const std::vector<FieldDesc>& fields_in, FieldState* d_state, FieldState* h_state, double* d_hist,
                  int hist_len, double tol, int window, double omega, int reunit_every, int abs_cap,
                  int check_every, bool fresh, cudaStream_t stream, bool solve32) {
    const int prec = sizeof(T) == 8 ? MCG_F64 : MCG_F32;
    const int NT = sweep_block(prec);
    const int SPB = sweep_sites_per_block(prec);
    const int nf = (int)fields_in.size();
    std::vector<FieldDesc> fields = fields_in;
    int total = 0;
    for (auto& fd : fields) {
        fd.nblk = (fd.geo.vh + SPB - 1) / SPB;
        fd.blk0 = total;
        total += fd.nblk;
    }
    int rc = 0;
    FieldDesc* d_desc = (FieldDesc*)scratch_device("fix.desc", sizeof(FieldDesc) * nf, &rc);
    if (rc) return rc;
    double* d_partial = (double*)scratch_device("fix.partial", sizeof(double) * total * (SPB / 32), &rc);
    if (rc) return rc;
    FieldDesc* h_desc = (FieldDesc*)scratch_host("fix.desc", sizeof(FieldDesc) * nf, &rc);
    if (rc) return rc;
    // the previous call may still read the pinned staging buffer
    MCG_CK(cudaStreamSynchronize(stream));
    std::copy(fields.begin(), fields.end(), h_desc);
    MCG_CK(cudaMemcpyAsync(d_desc, h_desc, sizeof(FieldDesc) * nf, cudaMemcpyHostToDevice, stream));
    // per-field phase caps
    MCG_CK(cudaMemcpyAsync(h_state, d_state, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost, stream));
    MCG_CK(cudaStreamSynchronize(stream));
    int min_sweep = 1 << 30;
    for (int f = 0; f < nf; ++f) {
        if (fresh) {
            h_state[f].sweep = 0;
            h_state[f].fallbacks = 0;
        }
        h_state[f].max_sweeps = abs_cap;
        h_state[f].done = 0;
        min_sweep = std::min(min_sweep, h_state[f].sweep);
    }
    const int phase_len = abs_cap - min_sweep;
    MCG_CK(cudaMemcpyAsync(d_state, h_state, sizeof(FieldState) * nf, cudaMemcpyHostToDevice, stream));

    SweepBatch bt;
    bt.desc = d_desc;
    bt.nf = nf;
    bt.total_blocks = total;
    bt.state = d_state;
    bt.partial = d_partial;
    bt.ppb = SPB / 32;
    bt.R_hist = d_hist;
    bt.hist_len = hist_len;
    bt.tol = tol;
    bt.window = std::max(1, std::min(window, kRing - 1));
    bt.reunit_every = reunit_every;
    bt.omega = omega;
    bt.solve32 = solve32 ? 1 : 0;

    if ((rc = prepare_halfsweep<T>(NT))) return rc;

    k_functional<T><<<total, SPB, 0, stream>>>(bt);
    k_finalize<<<nf, 256, 0, stream>>>(bt, fresh ? 1 : 2);
    MCG_CK(cudaGetLastError());
    note_launches(2);
    if (phase_len <= 0) {
        MCG_CK(cudaMemcpyAsync(h_state, d_state, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost, stream));
        MCG_CK(cudaStreamSynchronize(stream));
        return 0;
    }

    // graph of one chunk of sweeps, captured on the library's own stream
    const int chunk = std::max(1, std::min(check_every, phase_len));
    cudaStream_t cs = capture_stream(&rc);
    if (rc) return rc;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MCG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    for (int i = 0; i < chunk; ++i) enqueue_sweep<T>(bt, NT, SPB, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ce, "cudaGraphInstantiate");
    }
    const int nodes_per_chunk = chunk * ((sizeof(T) == 8 && reunit_every > 0) ? 4 : 3);
    const int max_chunks = (phase_len + chunk - 1) / chunk + 1;
    int status = 0;
    // phase timing (instrumentation): GPU time of the chunk graphs and the
    // site-updates they performed
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    const bool timed = cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess;
    std::vector<int> sw0(nf);
    for (int f = 0; f < nf; ++f) sw0[f] = h_state[f].sweep;
    for (int c = 0; c < max_chunks; ++c) {
        if (timed) cudaEventRecord(t0, stream);
        ce = cudaGraphLaunch(exec, stream);
        if (ce != cudaSuccess) {
            status = cuda_fail(ce, "cudaGraphLaunch");
            break;
        }
        if (timed) cudaEventRecord(t1, stream);
        note_launches(nodes_per_chunk);
        ce = cudaMemcpyAsync(h_state, d_state, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) {
            status = cuda_fail(ce, "sweep chunk");
            break;
        }
        if (timed) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            long long su = 0;
            for (int f = 0; f < nf; ++f) {
                su += (long long)(h_state[f].sweep - sw0[f]) * 2LL * fields[f].geo.vh;
                sw0[f] = h_state[f].sweep;
            }
            note_phase(sizeof(T) == 8 ? MCG_F64 : MCG_F32, ms, su);
        }
        bool all = true;
        for (int f = 0; f < nf; ++f) all = all && h_state[f].done != 0;
        if (all) break;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return status;
}

template <typename T>
int time_halfsweep(void* U, void* G, const Geom& g, int parity, int nreps, int flush_l2, float* ms,
                   cudaStream_t stream) {
    const int prec = sizeof(T) == 8 ? MCG_F64 : MCG_F32;
    const int NT = sweep_block(prec);
    const int SPB = sweep_sites_per_block(prec);
    int rc = 0;
    FieldDesc fd;
    fd.U = U;
    fd.G = G;
    fd.geo = g;
    fd.blk0 = 0;
    fd.nblk = (g.vh + SPB - 1) / SPB;
    fd.norm = 1.0 / (9.0 * 8.0 * g.vh);
    FieldDesc* d_desc = (FieldDesc*)scratch_device("time.desc", sizeof(FieldDesc), &rc);
    if (rc) return rc;
    FieldState* d_state = (FieldState*)scratch_device("time.state", sizeof(FieldState), &rc);
    if (rc) return rc;
    double* d_partial = (double*)scratch_device("time.partial", sizeof(double) * fd.nblk * (SPB / 32), &rc);
    if (rc) return rc;
    void* flush = nullptr;
    const size_t flush_bytes = (size_t)256 << 20;
    if (flush_l2) {
        flush = scratch_device("time.flush", flush_bytes, &rc);
        if (rc) return rc;
    }
    MCG_CK(cudaMemcpyAsync(d_desc, &fd, sizeof fd, cudaMemcpyHostToDevice, stream));
    MCG_CK(cudaMemsetAsync(d_state, 0, sizeof(FieldState), stream));
    SweepBatch bt;
    bt.desc = d_desc;
    bt.nf = 1;
    bt.total_blocks = fd.nblk;
    bt.state = d_state;
    bt.partial = d_partial;
    bt.ppb = SPB / 32;
    bt.R_hist = nullptr;
    bt.hist_len = 0;
    bt.tol = 0;
    bt.window = 1;
    bt.reunit_every = 0;
    bt.omega = 1.0;
    bt.solve32 = 0;
    if ((rc = prepare_halfsweep<T>(NT))) return rc;
    cudaEvent_t e0, e1;
    MCG_CK(cudaEventCreate(&e0));
    MCG_CK(cudaEventCreate(&e1));
    double total = 0.0;
    for (int r = 0; r < nreps; ++r) {
        if (flush) {
            cudaMemsetAsync(flush, r & 0xff, flush_bytes, stream);
        }
        cudaEventRecord(e0, stream);
        launch_halfsweep<T>(NT, parity != 0, bt, parity, fd.nblk, stream);
        cudaEventRecord(e1, stream);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(ce, "time_halfsweep");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        total += t;
    }
    note_launches(nreps);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MCG_CK(cudaGetLastError());
    *ms = (float)(total / std::max(1, nreps));
    return 0;
}

int run_anneal(void* U, void* G, const Geom& g, int nfields, const double* T, int nsweeps, long long first_sweep,
               int nhit, double eps, unsigned long long seed, long long* accepted_host, cudaStream_t st) {
    constexpr int NT = 128;
    const size_t smem = halfsweep_smem_f64(NT);
    int rc = 0;
    // per device and cheap: raised on every call
    if ((rc = raise_smem(k_anneal_halfsweep<NT>, smem))) return rc;
    unsigned long long* d_acc =
        (unsigned long long*)scratch_device("anneal.acc", sizeof(unsigned long long) * nfields, &rc);
    if (rc) return rc;
    unsigned long long* h_acc =
        (unsigned long long*)scratch_host("anneal.acc", sizeof(unsigned long long) * nfields, &rc);
    if (rc) return rc;
    MCG_CK(cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * nfields, st));
    AnnealArgs an;
    an.U = (cplx<double>*)U;
    an.G = (cplx<double>*)G;
    an.g = g;
    an.nhit = nhit;
    an.eps = eps;
    an.seed = seed;
    an.accepted = d_acc;
    const dim3 grid((g.vh + NT - 1) / NT, nfields);
    for (int k = 0; k < nsweeps; ++k) {
        an.T = T[k];
        an.sweep = first_sweep + k;
        for (int parity = 0; parity < 2; ++parity) k_anneal_halfsweep<NT><<<grid, NT, smem, st>>>(an, parity);
        MCG_CK(cudaGetLastError());
    }
    note_launches(2LL * nsweeps);
    if ((rc = launch_reunitarise(U, 0, MCG_F64, g, nfields, st))) return rc;
    if ((rc = launch_reunitarise(G, 1, MCG_F64, g, nfields, st))) return rc;
    MCG_CK(cudaMemcpyAsync(h_acc, d_acc, sizeof(unsigned long long) * nfields, cudaMemcpyDeviceToHost, st));
    MCG_CK(cudaStreamSynchronize(st));
    if (accepted_host)
        for (int f = 0; f < nfields; ++f) accepted_host[f] = (long long)h_acc[f];
    return 0;
}

template int time_halfsweep<float>(void*, void*, const Geom&, int, int, int, float*, cudaStream_t);
template int time_halfsweep<double>(void*, void*, const Geom&, int, int, int, float*, cudaStream_t);

template int run_fix_phase<float>(const std::vector<FieldDesc>&, FieldState*, FieldState*, double*, int, double,
                                  int, double, int, int, int, bool, cudaStream_t, bool);
template int run_fix_phase<double>(const std::vector<FieldDesc>&, FieldState*, FieldState*, double*, int, double,
                                   int, double, int, int, int, bool, cudaStream_t, bool);

}  // namespace mcg
