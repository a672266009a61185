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
