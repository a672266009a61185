// Stout and over-improved stout smearing (Sec. II.B; parameters of Sec. III).
// One thread per link; all links of a step are updated from the old field
// (out of place).  Staple weights of the over-improved action: (5 - 2 eps)/3
// on the plaquette staples and -(1 - eps)/12 on the rectangle staples;
// eps = 1 gives plain stout smearing.
//
// exp(iQ) for traceless Hermitian Q uses the Cayley-Hamilton closed form of
// Morningstar and Peardon (2004): exp(iQ) = f0 + f1 Q + f2 Q^2 with f_j from
// the invariants c0 = det Q, c1 = tr Q^2 / 2 (written here from that
// derivation); for tiny Q the power series reduced by Q^3 = c1 Q + c0 is used.
#include <cuda_runtime.h>

#include "mcg_common.cuh"
#include "mcg_internal.h"

namespace mcg {

constexpr int ST = 128;  // threads per block

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <typename T>
__device__ __forceinline__ void load_at(const cplx<T>* __restrict__ U, const Geom& g, int mu, const int c[4], int d0,
                                        int d1, int d2, int d3, cplx<T>* m) {
    int q[4] = {wrapc(c[0] + d0, g.n[0]), wrapc(c[1] + d1, g.n[1]), wrapc(c[2] + d2, g.n[2]),
                wrapc(c[3] + d3, g.n[3])};
    const int p = (q[0] + q[1] + q[2] + q[3]) & 1;
    const int s = eo_index(g, q);
    load_link(U, g, mu, p, s, m);
}

// displacement helpers: unit vectors scaled and summed
struct Disp {
    int d[4];
};
__device__ __forceinline__ Disp dsp(int mu, int a, int nu, int b) {
    Disp r = {{0, 0, 0, 0}};
    r.d[mu] += a;
    r.d[nu] += b;
    return r;
}

template <typename T>
__device__ __forceinline__ void ld(const cplx<T>* U, const Geom& g, int dir, const int c[4], Disp d, cplx<T>* m) {
    load_at(U, g, dir, c, d.d[0], d.d[1], d.d[2], d.d[3], m);
}

template <typename T>
__device__ __forceinline__ void acc(cplx<T>* C, const cplx<T>* m, T w) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        C[e].x = fma(w, m[e].x, C[e].x);
        C[e].y = fma(w, m[e].y, C[e].y);
    }
}

template <typename T>
__device__ __forceinline__ void dagger_inplace(cplx<T>* a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        a[4 * i].y = -a[4 * i].y;
#pragma unroll
        for (int j = i + 1; j < 3; ++j) {
            const cplx<T> u = a[3 * i + j], v = a[3 * j + i];
            a[3 * i + j] = mk(v.x, -v.y);
            a[3 * j + i] = mk(u.x, -u.y);
        }
    }
}

// r = a^dag (r must not alias a)
template <typename T>
__device__ __forceinline__ void dagger(const cplx<T>* a, cplx<T>* r) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r[3 * i + j] = mk(a[3 * j + i].x, -a[3 * j + i].y);
}

// exp(iQ), Q traceless Hermitian
template <typename T>
__device__ __forceinline__ void exp_iQ(const cplx<T>* Q, cplx<T>* E) {
    cplx<T> Q2[9];
    m3_mul(Q, Q, Q2);
    const T c1 = T(0.5) * (Q2[0].x + Q2[4].x + Q2[8].x);
    T c0 = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c0 += Q2[3 * i + j].x * Q[3 * j + i].x - Q2[3 * i + j].y * Q[3 * j + i].y;
    c0 *= T(1.0 / 3.0);
    cplx<T> f0, f1, f2;
    const T small = sizeof(T) == 8 ? T(1e-4) : T(1e-3);
    if (c1 < small) {
        // sum_k (iQ)^k / k! with Q^k = a_k + b_k Q + d_k Q^2, Q^3 = c1 Q + c0
        T a = 1, b = 0, d = 0;  // Q^0
        f0 = mk(T(1), T(0));
        f1 = mk(T(0), T(0));
        f2 = mk(T(0), T(0));
        T fact = 1;
        for (int k = 1; k <= 14; ++k) {
            const T na = d * c0, nb = a + d * c1, nd = b;
            a = na;
            b = nb;
            d = nd;
            fact /= (T)k;
            // i^k
            const int r = k & 3;
            const T sr = (r == 0) ? T(1) : (r == 2 ? T(-1) : T(0));
            const T si = (r == 1) ? T(1) : (r == 3 ? T(-1) : T(0));
            f0.x += sr * a * fact;
            f0.y += si * a * fact;
            f1.x += sr * b * fact;
            f1.y += si * b * fact;
            f2.x += sr * d * fact;
            f2.y += si * d * fact;
        }
    } else {
        const bool neg = c0 < T(0);
        const T c0a = fabs(c0);
        const T c0max = T(2) * c1 * sqrt(c1 / T(3)) / T(3);
        const T th = acos(fmin(c0a / c0max, T(1)));
        const T u = sqrt(c1 / T(3)) * cos(th / T(3));
        const T w = sqrt(c1) * sin(th / T(3));
        const T u2 = u * u, w2 = w * w;
        const T cw = cos(w);
        const T xi0 = fabs(w) < T(0.05) ? T(1) - w2 / T(6) * (T(1) - w2 / T(20) * (T(1) - w2 / T(42))) : sin(w) / w;
        const cplx<T> e2iu = mk(cos(T(2) * u), sin(T(2) * u));
        const cplx<T> emiu = mk(cos(u), -sin(u));
        const cplx<T> h0 = cadd(cscale(e2iu, u2 - w2), cmul(emiu, mk(T(8) * u2 * cw, T(2) * u * (T(3) * u2 + w2) * xi0)));
        const cplx<T> h1 = csub(cscale(e2iu, T(2) * u), cmul(emiu, mk(T(2) * u * cw, -(T(3) * u2 - w2) * xi0)));
        const cplx<T> h2 = csub(e2iu, cmul(emiu, mk(cw, T(3) * u * xi0)));
        const T inv = T(1) / (T(9) * u2 - w2);
        f0 = cscale(h0, inv);
        f1 = cscale(h1, inv);
        f2 = cscale(h2, inv);
        if (neg) {  // f_j(-c0) = (-1)^j conj(f_j(c0))
            f0 = mk(f0.x, -f0.y);
            f1 = mk(-f1.x, f1.y);
            f2 = mk(f2.x, -f2.y);
        }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        cplx<T> v = cadd(cmul(f1, Q[e]), cmul(f2, Q2[e]));
        if (e % 4 == 0) v = cadd(v, f0);
        E[e] = v;
    }
}

template <typename T, bool RECT>
__global__ void __launch_bounds__(ST) k_smear_step(const cplx<T>* __restrict__ Uin, cplx<T>* __restrict__ Uout, Geom g,
                                                   int nfields, T rho, T cp, T cr) {
    const long long n = 8LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (8LL * g.vh));
    int r = (int)(id - (long long)f * 8 * g.vh);
    const int mu = r / (2 * g.vh);
    r -= mu * 2 * g.vh;
    const int p = r / g.vh, s = r - p * g.vh;
    const cplx<T>* U = Uin + (size_t)f * link_elems(g);
    int c[4];
    eo_coords(g, p, s, c);

    cplx<T> C[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) C[e] = mk(T(0), T(0));
    cplx<T> a[9], b[9], t[9], t2[9];
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        // upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        ld(U, g, nu, c, dsp(mu, 0, nu, 0), a);
        ld(U, g, mu, c, dsp(mu, 0, nu, 1), b);
        m3_mul(a, b, t);
        ld(U, g, nu, c, dsp(mu, 1, nu, 0), a);
        m3_mul_nd(t, a, t2);
        acc(C, t2, cp);
        // lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        ld(U, g, nu, c, dsp(mu, 0, nu, -1), a);
        ld(U, g, mu, c, dsp(mu, 0, nu, -1), b);
        m3_mul_dn(a, b, t);
        ld(U, g, nu, c, dsp(mu, 1, nu, -1), a);
        m3_mul(t, a, t2);
        acc(C, t2, cp);
        if (RECT) {
            // 1x2, up: U_nu(x) U_nu(x+nu) U_mu(x+2nu) U_nu(x+mu+nu)^dag U_nu(x+mu)^dag
            ld(U, g, nu, c, dsp(mu, 0, nu, 0), a);
            ld(U, g, nu, c, dsp(mu, 0, nu, 1), b);
            m3_mul(a, b, t);
            ld(U, g, mu, c, dsp(mu, 0, nu, 2), a);
            m3_mul(t, a, t2);
            ld(U, g, nu, c, dsp(mu, 1, nu, 1), a);
            m3_mul_nd(t2, a, t);
            ld(U, g, nu, c, dsp(mu, 1, nu, 0), a);
            m3_mul_nd(t, a, t2);
            acc(C, t2, cr);
            // 1x2, down: U_nu(x-nu)^dag U_nu(x-2nu)^dag U_mu(x-2nu) U_nu(x-2nu+mu) U_nu(x-nu+mu)
            ld(U, g, nu, c, dsp(mu, 0, nu, -2), a);
            ld(U, g, nu, c, dsp(mu, 0, nu, -1), b);
            m3_mul(a, b, t);  // U_nu(x-2nu) U_nu(x-nu)
            ld(U, g, mu, c, dsp(mu, 0, nu, -2), a);
            m3_mul_dn(t, a, t2);  // (..)^dag U_mu(x-2nu)
            ld(U, g, nu, c, dsp(mu, 1, nu, -2), a);
            m3_mul(t2, a, t);
            ld(U, g, nu, c, dsp(mu, 1, nu, -1), a);
            m3_mul(t, a, t2);
            acc(C, t2, cr);
            // 2x1 forward, up: U_nu(x) U_mu(x+nu) U_mu(x+mu+nu) U_nu(x+2mu)^dag U_mu(x+mu)^dag
            ld(U, g, nu, c, dsp(mu, 0, nu, 0), a);
            ld(U, g, mu, c, dsp(mu, 0, nu, 1), b);
            m3_mul(a, b, t);
            ld(U, g, mu, c, dsp(mu, 1, nu, 1), a);
            m3_mul(t, a, t2);
            ld(U, g, nu, c, dsp(mu, 2, nu, 0), a);
            m3_mul_nd(t2, a, t);
            ld(U, g, mu, c, dsp(mu, 1, nu, 0), a);
            m3_mul_nd(t, a, t2);
            acc(C, t2, cr);
            // 2x1 forward, down: U_nu(x-nu)^dag U_mu(x-nu) U_mu(x-nu+mu) U_nu(x-nu+2mu) U_mu(x+mu)^dag
            ld(U, g, nu, c, dsp(mu, 0, nu, -1), a);
            ld(U, g, mu, c, dsp(mu, 0, nu, -1), b);
            m3_mul_dn(a, b, t);
            ld(U, g, mu, c, dsp(mu, 1, nu, -1), a);
            m3_mul(t, a, t2);
            ld(U, g, nu, c, dsp(mu, 2, nu, -1), a);
            m3_mul(t2, a, t);
            ld(U, g, mu, c, dsp(mu, 1, nu, 0), a);
            m3_mul_nd(t, a, t2);
            acc(C, t2, cr);
            // 2x1 backward, up: U_mu(x-mu)^dag U_nu(x-mu) U_mu(x-mu+nu) U_mu(x+nu) U_nu(x+mu)^dag
            ld(U, g, mu, c, dsp(mu, -1, nu, 0), a);
            ld(U, g, nu, c, dsp(mu, -1, nu, 0), b);
            m3_mul_dn(a, b, t);
            ld(U, g, mu, c, dsp(mu, -1, nu, 1), a);
            m3_mul(t, a, t2);
            ld(U, g, mu, c, dsp(mu, 0, nu, 1), a);
            m3_mul(t2, a, t);
            ld(U, g, nu, c, dsp(mu, 1, nu, 0), a);
            m3_mul_nd(t, a, t2);
            acc(C, t2, cr);
            // 2x1 backward, down: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_mu(x-nu) U_nu(x-nu+mu)
            ld(U, g, nu, c, dsp(mu, -1, nu, -1), a);
            ld(U, g, mu, c, dsp(mu, -1, nu, 0), b);
            m3_mul(a, b, t);  // U_nu(x-mu-nu) U_mu(x-mu)
            ld(U, g, mu, c, dsp(mu, -1, nu, -1), a);
            m3_mul_dn(t, a, t2);
            ld(U, g, mu, c, dsp(mu, 0, nu, -1), a);
            m3_mul(t2, a, t);
            ld(U, g, nu, c, dsp(mu, 1, nu, -1), a);
            m3_mul(t, a, t2);
            acc(C, t2, cr);
        }
    }
    // Omega = rho C U^dag; Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega)
    cplx<T> u[9], Om[9], Q[9], E[9];
    load_link(U, g, mu, p, s, u);
#pragma unroll
    for (int e = 0; e < 9; ++e) C[e] = cscale(C[e], rho);
    m3_mul_nd(C, u, Om);
    T trd = T(0);  // tr(Om^dag - Om) is purely imaginary: i * trd
#pragma unroll
    for (int i = 0; i < 3; ++i) trd += -T(2) * Om[4 * i].y;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // D_ij = conj(Om_ji) - Om_ij ; Q_ij = (i/2) D_ij
            const cplx<T> d = mk(Om[3 * j + i].x - Om[3 * i + j].x, -Om[3 * j + i].y - Om[3 * i + j].y);
            Q[3 * i + j] = mk(-T(0.5) * d.y, T(0.5) * d.x);
        }
    // - (i/6) * (i trd) = trd / 6 on the diagonal
#pragma unroll
    for (int i = 0; i < 3; ++i) Q[4 * i].x += trd / T(6);
    exp_iQ(Q, E);
    m3_mul(E, u, a);
    store_link(Uout + (size_t)f * link_elems(g), g, mu, p, s, a);
}

int run_smear(const void* Uin, void* Uout, int prec, const Geom& g, int nfields, double rho, double eps, int n,
              cudaStream_t st) {
    const size_t bytes = (prec == MCG_F64 ? 16 : 8) * link_elems(g) * (size_t)nfields;
    if (n <= 0) {
        MCG_CK(cudaMemcpyAsync(Uout, Uin, bytes, cudaMemcpyDeviceToDevice, st));
        return 0;
    }
    int rc = 0;
    void* tmp = nullptr;
    if (n >= 2) {
        tmp = scratch_device("smear.tmp", bytes, &rc);
        if (rc) return rc;
    }
    const double cp = (5.0 - 2.0 * eps) / 3.0, cr = -(1.0 - eps) / 12.0;
    const bool rect = cr != 0.0;
    const long long nthreads = 8LL * g.vh * nfields;
    const int nb = (int)((nthreads + ST - 1) / ST);
    const void* src = Uin;
    for (int k = 0; k < n; ++k) {
        void* dst = ((n - 1 - k) % 2 == 0) ? Uout : tmp;
        if (prec == MCG_F64) {
            if (rect)
                k_smear_step<double, true><<<nb, ST, 0, st>>>((const cplx<double>*)src, (cplx<double>*)dst, g, nfields,
                                                              rho, cp, cr);
            else
                k_smear_step<double, false><<<nb, ST, 0, st>>>((const cplx<double>*)src, (cplx<double>*)dst, g,
                                                               nfields, rho, cp, cr);
        } else {
            if (rect)
                k_smear_step<float, true><<<nb, ST, 0, st>>>((const cplx<float>*)src, (cplx<float>*)dst, g, nfields,
                                                             (float)rho, (float)cp, (float)cr);
            else
                k_smear_step<float, false><<<nb, ST, 0, st>>>((const cplx<float>*)src, (cplx<float>*)dst, g, nfields,
                                                              (float)rho, (float)cp, (float)cr);
        }
        MCG_CK(cudaGetLastError());
        note_launches(1);
        src = dst;
    }
    return 0;
}

}  // namespace mcg

// ===========================================================================
// Differentiation through smearing and of the MCG functional (not in the
// paper: the training pattern that differentiates the method).
// Matrix-gradient convention: for a real loss L of a link U,
// G = dL/dRe U + i dL/dIm U, so dL = Re tr(G^dag dU); in the SoA layout this
// is exactly the (re, im) pair a real-view autograd gradient holds.
// ===========================================================================
namespace mcg {

// Frechet derivative of exp at X in direction A, L(X, A), as the upper-right
// block of exp([[X, A], [0, X]]): Taylor recurrence on the blocks
// (p_{k+1} = p_k X / (k+1), s_{k+1} = (s_k X + p_k A) / (k+1)) after scaling
// by 2^-s, then s squarings [E, L] -> [E^2, E L + L E].
__device__ void frechet_exp(const cplx<double>* X, const cplx<double>* A, cplx<double>* L) {
    double nrm = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) nrm += cnorm2(X[e]);
    nrm = sqrt(nrm);
    int s = 0;
    while (nrm > 0.5 && s < 30) {
        nrm *= 0.5;
        ++s;
    }
    const double sc = ldexp(1.0, -s);
    cplx<double> Xs[9], As[9], p[9], q[9], E[9], t[9], t2[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        Xs[e] = cscale(X[e], sc);
        As[e] = cscale(A[e], sc);
        p[e] = mk((e % 4) == 0 ? 1.0 : 0.0, 0.0);
        q[e] = mk(0.0, 0.0);
        E[e] = p[e];
        L[e] = q[e];
    }
#pragma unroll 1
    for (int k = 1; k <= 18; ++k) {
        const double inv = 1.0 / k;
        m3_mul(q, Xs, t);   // s_k X
        m3_mul(p, As, t2);  // p_k A
#pragma unroll
        for (int e = 0; e < 9; ++e) q[e] = cscale(cadd(t[e], t2[e]), inv);
        m3_mul(p, Xs, t);
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            p[e] = cscale(t[e], inv);
            E[e] = cadd(E[e], p[e]);
            L[e] = cadd(L[e], q[e]);
        }
    }
#pragma unroll 1
    for (int r = 0; r < s; ++r) {
        m3_mul(E, L, t);
        m3_mul(L, E, t2);
#pragma unroll
        for (int e = 0; e < 9; ++e) L[e] = cadd(t[e], t2[e]);
        m3_mul(E, E, t);
#pragma unroll
        for (int e = 0; e < 9; ++e) E[e] = t[e];
    }
}

// One factor of a staple path: link direction (0: mu, 1: nu), displacement
// (dm along mu, dn along nu) of its site from x, daggered or not.
struct PathFactor {
    signed char dir, dm, dn, dag;
};
// The 8 staple shapes per nu != mu: two plaquette staples, then the six
// rectangle staples (1x2 up/down, 2x1 forward up/down, 2x1 backward up/down),
// each a path from x to x + mu.
__constant__ PathFactor c_paths[8][5] = {
    {{1, 0, 0, 0}, {0, 0, 1, 0}, {1, 1, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {1, 1, -1, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{1, 0, 0, 0}, {1, 0, 1, 0}, {0, 0, 2, 0}, {1, 1, 1, 1}, {1, 1, 0, 1}},
    {{1, 0, -1, 1}, {1, 0, -2, 1}, {0, 0, -2, 0}, {1, 1, -2, 0}, {1, 1, -1, 0}},
    {{1, 0, 0, 0}, {0, 0, 1, 0}, {0, 1, 1, 0}, {1, 2, 0, 1}, {0, 1, 0, 1}},
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {0, 1, -1, 0}, {1, 2, -1, 0}, {0, 1, 0, 1}},
    {{0, -1, 0, 1}, {1, -1, 0, 0}, {0, -1, 1, 0}, {0, 0, 1, 0}, {1, 1, 0, 1}},
    {{0, -1, 0, 1}, {1, -1, -1, 1}, {0, -1, -1, 0}, {0, 0, -1, 0}, {1, 1, -1, 0}},
};

__device__ __forceinline__ int factor_link(const Geom& g, const int c[4], int mu, int nu, PathFactor f, int* p_out) {
    int q[4] = {c[0], c[1], c[2], c[3]};
    q[mu] = wrapc(q[mu] + f.dm, g.n[mu]);
    q[nu] = wrapc(q[nu] + f.dn, g.n[nu]);
    *p_out = (q[0] + q[1] + q[2] + q[3]) & 1;
    return eo_index(g, q);
}

__device__ __forceinline__ void atomic_add_link(double* __restrict__ G, const Geom& g, int dir, int p, int s,
                                                const cplx<double>* m, bool dag) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const cplx<double> v = dag ? mk(m[3 * j + i].x, -m[3 * j + i].y) : m[3 * i + j];
            double* dst = G + 2 * lidx(g, dir, p, 3 * i + j, s);
            atomicAdd(dst, v.x);
            atomicAdd(dst + 1, v.y);
        }
}

// Reverse-mode derivative of one smearing step U' = exp(iQ(U)) U (FP64).
// Gin must be zeroed; every contribution is added atomically.
__global__ void __launch_bounds__(ST) k_smear_step_backward(const cplx<double>* __restrict__ Uall,
                                                            const cplx<double>* __restrict__ Gout_all,
                                                            double* __restrict__ Gin_all, Geom g, int nfields,
                                                            double rho, double cp, double cr) {
    const long long n = 8LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (8LL * g.vh));
    int r = (int)(id - (long long)f * 8 * g.vh);
    const int mu = r / (2 * g.vh);
    r -= mu * 2 * g.vh;
    const int p = r / g.vh, s = r - p * g.vh;
    const cplx<double>* U = Uall + (size_t)f * link_elems(g);
    const cplx<double>* Gout = Gout_all + (size_t)f * link_elems(g);
    double* Gin = Gin_all + 2 * (size_t)f * link_elems(g);
    int c[4];
    eo_coords(g, p, s, c);
    const int npat = cr != 0.0 ? 8 : 2;

    cplx<double> u[9], go[9], C[9], a[9], b[9], t[9];
    load_link(U, g, mu, p, s, u);
    load_link(Gout, g, mu, p, s, go);
    // staple sum C = rho * sum_w w * W
#pragma unroll
    for (int e = 0; e < 9; ++e) C[e] = mk(0.0, 0.0);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        for (int k = 0; k < npat; ++k) {
            const int nf = k < 2 ? 3 : 5;
            const double w = k < 2 ? cp : cr;
#pragma unroll 1
            for (int j = 0; j < nf; ++j) {
                const PathFactor fct = c_paths[k][j];
                int pp;
                const int ss = factor_link(g, c, mu, nu, fct, &pp);
                load_link(U, g, fct.dir ? nu : mu, pp, ss, b);
                if (fct.dag) dagger_inplace(b);
                if (j == 0) {
#pragma unroll
                    for (int e = 0; e < 9; ++e) a[e] = b[e];
                } else {
                    m3_mul(a, b, t);
#pragma unroll
                    for (int e = 0; e < 9; ++e) a[e] = t[e];
                }
            }
            acc(C, a, w);
        }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) C[e] = cscale(C[e], rho);
    // Q, E = exp(iQ)
    cplx<double> Om[9], Q[9], E[9], X[9], B[9], K[9], Y[9];
    m3_mul_nd(C, u, Om);
    double trd = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) trd += -2.0 * Om[4 * i].y;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const cplx<double> d = mk(Om[3 * j + i].x - Om[3 * i + j].x, -Om[3 * j + i].y - Om[3 * i + j].y);
            Q[3 * i + j] = mk(-0.5 * d.y, 0.5 * d.x);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i) Q[4 * i].x += trd / 6.0;
    exp_iQ(Q, E);
    // direct term E^dag Gout
    m3_mul_dn(E, go, t);
    atomic_add_link(Gin, g, mu, p, s, t, false);
    // exp adjoint: B = L(iQ, U Gout^dag); K = traceless anti-Hermitian part
#pragma unroll
    for (int e = 0; e < 9; ++e) X[e] = mk(-Q[e].y, Q[e].x);
    m3_mul_nd(u, go, a);
    frechet_exp(X, a, B);
    double tki = 0.0, tkr = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            K[3 * i + j] = mk(0.5 * (B[3 * i + j].x - B[3 * j + i].x), 0.5 * (B[3 * i + j].y + B[3 * j + i].y));
            if (i == j) {
                tkr += K[3 * i + j].x;
                tki += K[3 * i + j].y;
            }
        }
#pragma unroll
    for (int i = 0; i < 3; ++i) K[4 * i] = mk(K[4 * i].x - tkr / 3.0, K[4 * i].y - tki / 3.0);
    // Omega = C U^dag: K C on this link, rho U^dag K scattered over the staples
    m3_mul(K, C, t);
    atomic_add_link(Gin, g, mu, p, s, t, false);
    m3_mul_dn(u, K, Y);
#pragma unroll
    for (int e = 0; e < 9; ++e) Y[e] = cscale(Y[e], rho);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        for (int k = 0; k < npat; ++k) {
            const int nf = k < 2 ? 3 : 5;
            const double w = k < 2 ? cp : cr;
            // Z_j = F_{j+1} ... F_{nf-1} (w Y) F_0 ... F_{j-1} for each factor j;
            // factors are re-loaded (from L1) rather than held in per-thread
            // arrays, which keeps this kernel free of dynamically indexed
            // local memory
#pragma unroll 1
            for (int j = 0; j < nf; ++j) {
                cplx<double> Z[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) Z[e] = cscale(Y[e], w);
#pragma unroll 1
                for (int m = nf - 1; m > j; --m) {
                    const PathFactor fm = c_paths[k][m];
                    int pm;
                    const int sm = factor_link(g, c, mu, nu, fm, &pm);
                    load_link(U, g, fm.dir ? nu : mu, pm, sm, b);
                    if (fm.dag) dagger_inplace(b);
                    m3_mul(b, Z, t);
#pragma unroll
                    for (int e = 0; e < 9; ++e) Z[e] = t[e];
                }
#pragma unroll 1
                for (int m = 0; m < j; ++m) {
                    const PathFactor fm = c_paths[k][m];
                    int pm;
                    const int sm = factor_link(g, c, mu, nu, fm, &pm);
                    load_link(U, g, fm.dir ? nu : mu, pm, sm, b);
                    if (fm.dag) dagger_inplace(b);
                    m3_mul(Z, b, t);
#pragma unroll
                    for (int e = 0; e < 9; ++e) Z[e] = t[e];
                }
                const PathFactor fct = c_paths[k][j];
                int pj;
                const int sj = factor_link(g, c, mu, nu, fct, &pj);
                // factor U: gradient += Z^dag; factor U^dag: gradient += Z
                atomic_add_link(Gin, g, fct.dir ? nu : mu, pj, sj, Z, !fct.dag);
            }
        }
    }
}

// G = 2 tr(U) 1 per link: the matrix gradient of R = sum |tr U|^2 (FP64 out).
template <typename T>
__global__ void __launch_bounds__(256) k_functional_matrix_grad(const cplx<T>* __restrict__ U, double* __restrict__ G,
                                                                Geom g, int nfields) {
    const long long n = 8LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (8LL * g.vh));
    int r = (int)(id - (long long)f * 8 * g.vh);
    const int mu = r / (2 * g.vh);
    r -= mu * 2 * g.vh;
    const int p = r / g.vh, s = r - p * g.vh;
    const cplx<T>* Uf = U + (size_t)f * link_elems(g);
    double* Gf = G + 2 * (size_t)f * link_elems(g);
    const cplx<T> d0 = Uf[lidx(g, mu, p, 0, s)], d1 = Uf[lidx(g, mu, p, 4, s)], d2 = Uf[lidx(g, mu, p, 8, s)];
    const double tr = 2.0 * ((double)d0.x + (double)d1.x + (double)d2.x);
    const double ti = 2.0 * ((double)d0.y + (double)d1.y + (double)d2.y);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const bool diag = (e % 4) == 0;
        Gf[2 * lidx(g, mu, p, e, s)] = diag ? tr : 0.0;
        Gf[2 * lidx(g, mu, p, e, s) + 1] = diag ? ti : 0.0;
    }
}

// tr(lambda_a M) for the eight Gell-Mann matrices (tr(lambda_a lambda_b) = 2 delta_ab)
__device__ __forceinline__ void gellmann_traces(const cplx<double>* M, cplx<double>* t) {
    t[0] = cadd(M[3], M[1]);                                  // lambda_1
    t[1] = mk(M[3].y - M[1].y, M[1].x - M[3].x);              // -i M10 + i M01
    t[2] = csub(M[0], M[4]);                                  // lambda_3
    t[3] = cadd(M[6], M[2]);                                  // lambda_4
    t[4] = mk(M[6].y - M[2].y, M[2].x - M[6].x);              // -i M20 + i M02
    t[5] = cadd(M[7], M[5]);                                  // lambda_6
    t[6] = mk(M[7].y - M[5].y, M[5].x - M[7].x);              // -i M21 + i M12
    const double s3 = 0.57735026918962576;                    // 1/sqrt(3)
    t[7] = mk(s3 * (M[0].x + M[4].x - 2.0 * M[8].x), s3 * (M[0].y + M[4].y - 2.0 * M[8].y));
}

// dR/d eps_a(x) for Omega(x) -> exp(i eps lambda_a / 2) Omega(x):
// sum_mu Re[conj(t_f) i tr(lambda_a U_mu(x))] - Re[conj(t_b) i tr(lambda_a U_mu(x-mu))]
// (the factor 2 of |t|^2 cancels the 1/2 of T_a = lambda_a / 2).
// grad: [field][lexicographic site][8].
template <typename T>
__global__ void __launch_bounds__(256) k_grad_R(const cplx<T>* __restrict__ U, double* __restrict__ grad, Geom g,
                                                int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    const cplx<T>* Uf = U + (size_t)f * link_elems(g);
    int c[4];
    eo_coords(g, p, s, c);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int mu = 0; mu < 4; ++mu) {
        const int sb = eo_neighbor(g, c, mu, -1);
        for (int side = 0; side < 2; ++side) {
            cplx<double> m[9], tg[8];
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                const cplx<T> v = side == 0 ? Uf[lidx(g, mu, p, e, s)] : Uf[lidx(g, mu, p ^ 1, e, sb)];
                m[e] = mk((double)v.x, (double)v.y);
            }
            const cplx<double> tr = cadd(cadd(m[0], m[4]), m[8]);
            gellmann_traces(m, tg);
            const double sgn = side == 0 ? 1.0 : -1.0;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                // Re[conj(tr) * i * tg] = tr.x * (-tg.y) + tr.y * tg.x
                acc[a] += sgn * (tr.y * tg[a].x - tr.x * tg[a].y);
            }
        }
    }
    const long long lex = (long long)c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * (c[2] + (long long)g.n[2] * c[3]));
    double* out = grad + ((size_t)f * 2 * g.vh + lex) * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) out[a] = acc[a];
}

// Ascent step, part 1: W(x) = exp(i alpha sum_a grad_a(x) lambda_a / 2) into
// scratch and Omega(x) <- W(x) Omega(x).
template <typename T>
__global__ void __launch_bounds__(256) k_ascent_gauge(const double* __restrict__ grad, double alpha,
                                                      cplx<T>* __restrict__ Gauge, cplx<T>* __restrict__ Wout, Geom g,
                                                      int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    int c[4];
    eo_coords(g, p, s, c);
    const long long lex = (long long)c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * (c[2] + (long long)g.n[2] * c[3]));
    const double* ga = grad + ((size_t)f * 2 * g.vh + lex) * 8;
    double h[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) h[a] = 0.5 * alpha * ga[a];
    // Q = sum_a h_a lambda_a (Hermitian, traceless)
    cplx<double> Q[9], E[9];
    const double s3 = 0.57735026918962576;
    Q[0] = mk(h[2] + s3 * h[7], 0.0);
    Q[4] = mk(-h[2] + s3 * h[7], 0.0);
    Q[8] = mk(-2.0 * s3 * h[7], 0.0);
    Q[1] = mk(h[0], -h[1]);
    Q[3] = mk(h[0], h[1]);
    Q[2] = mk(h[3], -h[4]);
    Q[6] = mk(h[3], h[4]);
    Q[5] = mk(h[5], -h[6]);
    Q[7] = mk(h[5], h[6]);
    exp_iQ(Q, E);
    cplx<T>* Gf = Gauge + (size_t)f * gauge_elems(g);
    cplx<T>* Wf = Wout + (size_t)f * gauge_elems(g);
    cplx<double> o[9], t[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const cplx<T> v = Gf[gidx(g, p, e, s)];
        o[e] = mk((double)v.x, (double)v.y);
    }
    m3_mul(E, o, t);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        Gf[gidx(g, p, e, s)] = mk((T)t[e].x, (T)t[e].y);
        Wf[gidx(g, p, e, s)] = mk((T)E[e].x, (T)E[e].y);
    }
}

int run_smear_step_backward(const void* U, const double* Gout, double* Gin, const Geom& g, int nfields, double rho,
                            double eps, cudaStream_t st) {
    const double cp = (5.0 - 2.0 * eps) / 3.0, cr = -(1.0 - eps) / 12.0;
    MCG_CK(cudaMemsetAsync(Gin, 0, 16 * link_elems(g) * (size_t)nfields, st));
    const long long n = 8LL * g.vh * nfields;
    k_smear_step_backward<<<(int)((n + ST - 1) / ST), ST, 0, st>>>((const cplx<double>*)U, (const cplx<double>*)Gout,
                                                                    Gin, g, nfields, rho, cp, cr);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int run_functional_matrix_grad(const void* U, int prec, double* G, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 8LL * g.vh * nfields;
    const int nb = (int)((n + 255) / 256);
    if (prec == MCG_F64)
        k_functional_matrix_grad<double><<<nb, 256, 0, st>>>((const cplx<double>*)U, G, g, nfields);
    else
        k_functional_matrix_grad<float><<<nb, 256, 0, st>>>((const cplx<float>*)U, G, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int run_grad_R(const void* U, int prec, double* grad, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    const int nb = (int)((n + 255) / 256);
    if (prec == MCG_F64)
        k_grad_R<double><<<nb, 256, 0, st>>>((const cplx<double>*)U, grad, g, nfields);
    else
        k_grad_R<float><<<nb, 256, 0, st>>>((const cplx<float>*)U, grad, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int run_ascent_step(void* U, void* G, const double* grad, double alpha, int prec, const Geom& g, int nfields,
                    cudaStream_t st) {
    int rc = 0;
    const size_t eb = prec == MCG_F64 ? 16 : 8;
    void* W = scratch_device("ascent.W", eb * gauge_elems(g) * nfields, &rc);
    if (rc) return rc;
    const long long n = 2LL * g.vh * nfields;
    const int nb = (int)((n + 255) / 256);
    if (prec == MCG_F64)
        k_ascent_gauge<double><<<nb, 256, 0, st>>>(grad, alpha, (cplx<double>*)G, (cplx<double>*)W, g, nfields);
    else
        k_ascent_gauge<float><<<nb, 256, 0, st>>>(grad, alpha, (cplx<float>*)G, (cplx<float>*)W, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return launch_apply_gauge(U, W, prec, g, nfields, st);
}

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_smear)

}  // namespace mcg
