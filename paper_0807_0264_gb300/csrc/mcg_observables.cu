// Observables on the center decomposition of a fixed field (Sec. III.D): the
// vortex-removed field U' = Z^dag U, the vortex-only field Z, and planar
// Wilson loops W(R, T) averaged over all translations and spatial axes.
#include <algorithm>
#include <vector>

#include "mcg_internal.h"

namespace mcg {

namespace {

constexpr int OT = 256;  // threads per block of the streaming kernels

inline int nblocks(long long n, int nt) { return (int)((n + nt - 1) / nt); }

// exp(2 pi i m / 3) as (cos, sin); the values for m = +-1 are the literals
// -1/2 and +-sqrt(3)/2
__device__ __forceinline__ void center_phase(int m, double& c, double& s) {
    c = m == 0 ? 1.0 : -0.5;
    s = m == 0 ? 0.0 : (m > 0 ? 0.8660254037844386 : -0.8660254037844386);
}

// conj(Z) u with products and sums rounded separately (no fused operations):
// re' = c re + s im, im' = c im - s re
__device__ __forceinline__ cplx<double> unphase(cplx<double> u, double c, double s) {
    return mk(__dadd_rn(__dmul_rn(c, u.x), __dmul_rn(s, u.y)), __dsub_rn(__dmul_rn(c, u.y), __dmul_rn(s, u.x)));
}
__device__ __forceinline__ cplx<float> unphase(cplx<float> u, double c, double s) {
    const float cf = (float)c, sf = (float)s;
    return mk(__fadd_rn(__fmul_rn(cf, u.x), __fmul_rn(sf, u.y)), __fsub_rn(__fmul_rn(cf, u.y), __fmul_rn(sf, u.x)));
}

// One thread per (field, parity, site): its 4 links.  Ur (may be null, may
// be U itself): Z^dag U; Zl (may be null): the center links Z * identity.
template <typename T>
__global__ void __launch_bounds__(OT) k_vortex_remove(const cplx<T>* U, const int8_t* __restrict__ Z, cplx<T>* Ur,
                                                      cplx<T>* __restrict__ Zl, Geom g, int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    const size_t lo = (size_t)f * link_elems(g);
    const int8_t* Zf = Z + (size_t)f * 8 * g.vh;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int m = Zf[(size_t)(mu * 2 + p) * g.vh + s];
        double c, sn;
        center_phase(m, c, sn);
        if (Ur) {
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                const size_t k = lo + lidx(g, mu, p, e, s);
                Ur[k] = unphase(U[k], c, sn);
            }
        }
        if (Zl) {
#pragma unroll
            for (int e = 0; e < 9; ++e)
                Zl[lo + lidx(g, mu, p, e, s)] = (e % 4 == 0) ? mk((T)c, (T)sn) : mk((T)0, (T)0);
        }
    }
}

// ---- Wilson loops -----------------------------------------------------------
// Line products S_mu^L(x) = U_mu(x) U_mu(x+mu) ... U_mu(x+(L-1)mu) are kept in
// lexicographic site order, one SoA array per matrix entry: L[e * V + x].
// Links are read from the even/odd field layout (in-parity index x / 2).

__device__ __forceinline__ void lex_coords(const Geom& g, int x, int c[4]) {
    c[0] = x % g.n[0];
    int r = x / g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
}
__device__ __forceinline__ int lex_index(const Geom& g, const int c[4]) {
    return c[0] + g.n[0] * (c[1] + g.n[1] * (c[2] + g.n[2] * c[3]));
}
// lexicographic index of x + k mu (k >= 0), periodic
__device__ __forceinline__ int lex_shift(const Geom& g, int x, int mu, int k) {
    int c[4];
    lex_coords(g, x, c);
    c[mu] = (c[mu] + k) % g.n[mu];
    return lex_index(g, c);
}

template <typename T>
__device__ __forceinline__ void load_field_link(const cplx<T>* __restrict__ U, const Geom& g, int x, int mu,
                                                cplx<T>* m) {
    int c[4];
    lex_coords(g, x, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = U[lidx(g, mu, p, e, x >> 1)];
}

template <typename T>
__device__ __forceinline__ void load_line(const cplx<T>* __restrict__ L, int V, int x, cplx<T>* m) {
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = L[(size_t)e * V + x];
}

// Lout(x) = Lin(x) U_mu(x + (len-1) mu); len == 1 copies the link (Lin unused)
template <typename T>
__global__ void __launch_bounds__(OT) k_line_extend(const cplx<T>* __restrict__ U, const cplx<T>* __restrict__ Lin,
                                                    cplx<T>* __restrict__ Lout, Geom g, int mu, int len) {
    const int V = 2 * g.vh;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    cplx<T> u[9], out[9];
    load_field_link(U, g, lex_shift(g, x, mu, len - 1), mu, u);
    if (len == 1) {
#pragma unroll
        for (int e = 0; e < 9; ++e) out[e] = u[e];
    } else {
        cplx<T> a[9];
        load_line(Lin, V, x, a);
        m3_mul(a, u, out);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) Lout[(size_t)e * V + x] = out[e];
}

// Per-block partial of sum over sites x and spatial axes i of
// (1/3) Re tr[ S_i^R(x) S_t^T(x+R i) (S_t^T(x) S_i^R(x+T t))^dag ].
// Si: the three spatial lines of length R; St: the temporal line of length T.
template <typename T>
__global__ void __launch_bounds__(OT) k_wilson_RT(const cplx<T>* __restrict__ Si, const cplx<T>* __restrict__ St,
                                                  Geom g, int R, int Tl, double* __restrict__ partial) {
    const int V = 2 * g.vh;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (x < V) {
        const int xt = lex_shift(g, x, 3, Tl);
        cplx<T> c[9];
        load_line(St, V, x, c);
#pragma unroll 1
        for (int i = 0; i < 3; ++i) {
            const cplx<T>* Li = Si + (size_t)i * 9 * V;
            cplx<T> s[9], a[9], b[9], X[9], Y[9];
            load_line(Li, V, x, s);
            load_line(St, V, lex_shift(g, x, i, R), a);
            load_line(Li, V, xt, b);
            m3_mul(s, a, X);  // S_i^R(x) S_t^T(x + R i)
            m3_mul(c, b, Y);  // S_t^T(x) S_i^R(x + T t)
            // tr(X Y^dag) = sum_jk X_jk conj(Y_jk)
            double re = 0.0;
#pragma unroll
            for (int e = 0; e < 9; ++e) re += (double)X[e].x * (double)Y[e].x + (double)X[e].y * (double)Y[e].y;
            acc += re / 3.0;
        }
    }
    __shared__ double red[OT / 32];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_sum_fixed(const double* __restrict__ partial, int n, double scale, double* __restrict__ out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partial[k];
    __shared__ double red[8];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) *out = tot * scale;
}

template <typename T>
int wilson_impl(const cplx<T>* U, const Geom& g, int nfields, int Rmax, int Tmax, double* W_host, cudaStream_t st) {
    const int V = 2 * g.vh;
    const size_t line = (size_t)9 * V;  // elements of one line field
    int rc = 0;
    cplx<T>* Lt = (cplx<T>*)scratch_device("wl.t", sizeof(cplx<T>) * line * Tmax, &rc);
    if (rc) return rc;
    cplx<T>* Ls = (cplx<T>*)scratch_device("wl.s", sizeof(cplx<T>) * line * 6, &rc);  // 3 axes x 2 buffers
    if (rc) return rc;
    const int nb = nblocks(V, OT);
    double* partial = (double*)scratch_device("wl.partial", sizeof(double) * nb, &rc);
    if (rc) return rc;
    double* d_W = (double*)scratch_device("wl.W", sizeof(double) * (size_t)nfields * Rmax * Tmax, &rc);
    if (rc) return rc;
    long long launches = 0;
    for (int f = 0; f < nfields; ++f) {
        const cplx<T>* Uf = U + (size_t)f * link_elems(g);
        for (int T_ = 1; T_ <= Tmax; ++T_) {
            k_line_extend<T><<<nb, OT, 0, st>>>(Uf, Lt + line * (T_ - 2 < 0 ? 0 : T_ - 2), Lt + line * (T_ - 1), g, 3,
                                                T_);
            ++launches;
        }
        for (int R = 1; R <= Rmax; ++R) {
            cplx<T>* cur = Ls + line * 3 * (R & 1);
            const cplx<T>* prev = Ls + line * 3 * ((R + 1) & 1);
            for (int i = 0; i < 3; ++i) {
                k_line_extend<T><<<nb, OT, 0, st>>>(Uf, prev + line * i, cur + line * i, g, i, R);
                ++launches;
            }
            for (int T_ = 1; T_ <= Tmax; ++T_) {
                k_wilson_RT<T><<<nb, OT, 0, st>>>(cur, Lt + line * (T_ - 1), g, R, T_, partial);
                k_sum_fixed<<<1, 256, 0, st>>>(partial, nb, 1.0 / (3.0 * V),
                                               d_W + ((size_t)f * Rmax + (R - 1)) * Tmax + (T_ - 1));
                launches += 2;
            }
        }
    }
    MCG_CK(cudaGetLastError());
    note_launches(launches);
    MCG_CK(cudaMemcpyAsync(W_host, d_W, sizeof(double) * (size_t)nfields * Rmax * Tmax, cudaMemcpyDeviceToHost, st));
    MCG_CK(cudaStreamSynchronize(st));
    return 0;
}

}  // namespace

int launch_vortex_remove(const void* U, const int8_t* Z, void* Ur, void* Zl, int prec, const Geom& g, int nfields,
                         cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    if (prec == MCG_F64)
        k_vortex_remove<double><<<nblocks(n, OT), OT, 0, st>>>((const cplx<double>*)U, Z, (cplx<double>*)Ur,
                                                               (cplx<double>*)Zl, g, nfields);
    else
        k_vortex_remove<float><<<nblocks(n, OT), OT, 0, st>>>((const cplx<float>*)U, Z, (cplx<float>*)Ur,
                                                              (cplx<float>*)Zl, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int compute_wilson_loops(const void* U, int prec, const Geom& g, int nfields, int Rmax, int Tmax, double* W_host,
                         cudaStream_t st) {
    if (prec == MCG_F64) return wilson_impl<double>((const cplx<double>*)U, g, nfields, Rmax, Tmax, W_host, st);
    return wilson_impl<float>((const cplx<float>*)U, g, nfields, Rmax, Tmax, W_host, st);
}

}  // namespace mcg
