// Observables on the center decomposition of a fixed field (Sec. III.A): the
// vortex-removed field U' = Z^dag U, the vortex-only field Z, and planar
// Wilson loops W(R, T) averaged over all translations and spatial axes.
#include <algorithm>
#include <array>
#include <cstdlib>
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

// ---- off-axis spatial sides -------------------------------------------------
// lexicographic index of x + (d0, d1, d2, d3), periodic, any signs
__device__ __forceinline__ int lex_offset(const Geom& g, int x, int d0, int d1, int d2, int d3) {
    int c[4];
    lex_coords(g, x, c);
    const int d[4] = {d0, d1, d2, d3};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] = ((c[mu] + d[mu]) % g.n[mu] + g.n[mu]) % g.n[mu];
    return lex_index(g, c);
}

// One step of a spatial path: the path so far ends at x + (o0, o1, o2);
// Pout(x) = Pin(x) U_axis(x + o) for a forward step, Pin(x) U_axis(x + o -
// axis)^dag for a backward one (first: Pin is the identity).
template <typename T>
__global__ void __launch_bounds__(OT) k_path_step(const cplx<T>* __restrict__ U, const cplx<T>* __restrict__ Pin,
                                                  cplx<T>* __restrict__ Pout, Geom g, int o0, int o1, int o2,
                                                  int axis, int sign, int first) {
    const int V = 2 * g.vh;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    const int back = sign < 0 ? 1 : 0;
    const int y = lex_offset(g, x, o0 - (axis == 0 ? back : 0), o1 - (axis == 1 ? back : 0),
                             o2 - (axis == 2 ? back : 0), 0);
    cplx<T> u[9], out[9];
    load_field_link(U, g, y, axis, u);
    if (back) {
        cplx<T> d[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) d[3 * i + j] = mk(u[3 * j + i].x, -u[3 * j + i].y);
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = d[e];
    }
    if (first) {
#pragma unroll
        for (int e = 0; e < 9; ++e) out[e] = u[e];
    } else {
        cplx<T> a[9];
        load_line(Pin, V, x, a);
        m3_mul(a, u, out);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) Pout[(size_t)e * V + x] = out[e];
}

// Per-block partial of sum over sites of
// (1/3) Re tr[ P(x) S_t^T(x + r) (S_t^T(x) P(x + T t))^dag ].
template <typename T>
__global__ void __launch_bounds__(OT) k_wilson_path(const cplx<T>* __restrict__ P, const cplx<T>* __restrict__ St,
                                                    Geom g, int r0, int r1, int r2, int Tl,
                                                    double* __restrict__ partial) {
    const int V = 2 * g.vh;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (x < V) {
        cplx<T> p[9], a[9], b[9], c[9], X[9], Y[9];
        load_line(P, V, x, p);
        load_line(St, V, lex_offset(g, x, r0, r1, r2, 0), a);
        load_line(St, V, x, c);
        load_line(P, V, lex_offset(g, x, 0, 0, 0, Tl), b);
        m3_mul(p, a, X);
        m3_mul(c, b, Y);
        double re = 0.0;
#pragma unroll
        for (int e = 0; e < 9; ++e) re += (double)X[e].x * (double)Y[e].x + (double)X[e].y * (double)Y[e].y;
        acc = re / 3.0;
    }
    __shared__ double red[OT / 32];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// The distinct images of r under the 48 axis permutations with sign flips.
std::vector<std::array<int, 3>> cubic_images(const int* r) {
    std::vector<std::array<int, 3>> out;
    int p[3] = {0, 1, 2};
    std::sort(p, p + 3);
    do {
        for (int sg = 0; sg < 8; ++sg) {
            std::array<int, 3> v;
            for (int j = 0; j < 3; ++j) v[j] = r[p[j]] * (((sg >> j) & 1) ? -1 : 1);
            if (std::find(out.begin(), out.end(), v) == out.end()) out.push_back(v);
        }
    } while (std::next_permutation(p, p + 3));
    return out;
}

// Steps of the spatial path of r: each step along the axis with the largest
// deficit k |r_j| / L - n_j (ties to the lowest axis), towards sign(r_j).
void path_steps(const std::array<int, 3>& r, std::vector<int>& axis, std::vector<int>& sign) {
    const int L = std::abs(r[0]) + std::abs(r[1]) + std::abs(r[2]);
    int n[3] = {0, 0, 0};
    axis.clear();
    sign.clear();
    for (int k = 1; k <= L; ++k) {
        int best = -1;
        double bd = -1e300;
        for (int j = 0; j < 3; ++j) {
            if (n[j] >= std::abs(r[j])) continue;
            const double d = (double)k * std::abs(r[j]) / L - n[j];
            if (d > bd) {
                bd = d;
                best = j;
            }
        }
        axis.push_back(best);
        sign.push_back(r[best] > 0 ? 1 : -1);
        n[best]++;
    }
}

template <typename T>
int wilson_offaxis_impl(const cplx<T>* U, const Geom& g, int nfields, const int* vecs, int nvec, int Tmax,
                        double* W_host, cudaStream_t st) {
    const int V = 2 * g.vh;
    const size_t line = (size_t)9 * V;
    int rc = 0;
    cplx<T>* Lt = (cplx<T>*)scratch_device("wl.t", sizeof(cplx<T>) * line * Tmax, &rc);
    if (rc) return rc;
    cplx<T>* Pb = (cplx<T>*)scratch_device("wl.s", sizeof(cplx<T>) * line * 6, &rc);  // two path buffers
    if (rc) return rc;
    const int nb = nblocks(V, OT);
    double* partial = (double*)scratch_device("wl.partial", sizeof(double) * nb, &rc);
    if (rc) return rc;
    std::vector<std::vector<std::array<int, 3>>> imgs(nvec);
    size_t nimg_tot = 0;
    for (int v = 0; v < nvec; ++v) {
        imgs[v] = cubic_images(vecs + 3 * v);
        nimg_tot += imgs[v].size();
    }
    double* d_W = (double*)scratch_device("wl.Wimg", sizeof(double) * nimg_tot * Tmax, &rc);
    if (rc) return rc;
    std::vector<double> h_W(nimg_tot * Tmax);
    long long launches = 0;
    std::vector<int> axis, sign;
    for (int f = 0; f < nfields; ++f) {
        const cplx<T>* Uf = U + (size_t)f * link_elems(g);
        for (int T_ = 1; T_ <= Tmax; ++T_) {
            k_line_extend<T><<<nb, OT, 0, st>>>(Uf, Lt + line * (T_ - 2 < 0 ? 0 : T_ - 2), Lt + line * (T_ - 1), g, 3,
                                                T_);
            ++launches;
        }
        size_t q = 0;
        for (int v = 0; v < nvec; ++v)
            for (const auto& r : imgs[v]) {
                path_steps(r, axis, sign);
                int o[3] = {0, 0, 0};
                int cur = 0;
                for (size_t k = 0; k < axis.size(); ++k) {
                    k_path_step<T><<<nb, OT, 0, st>>>(Uf, Pb + line * cur, Pb + line * (1 - cur), g, o[0], o[1], o[2],
                                                      axis[k], sign[k], k == 0 ? 1 : 0);
                    ++launches;
                    o[axis[k]] += sign[k];
                    cur = 1 - cur;
                }
                for (int T_ = 1; T_ <= Tmax; ++T_) {
                    k_wilson_path<T><<<nb, OT, 0, st>>>(Pb + line * cur, Lt + line * (T_ - 1), g, r[0], r[1], r[2], T_,
                                                        partial);
                    k_sum_fixed<<<1, 256, 0, st>>>(partial, nb, 1.0 / V, d_W + q * Tmax + (T_ - 1));
                    launches += 2;
                }
                ++q;
            }
        MCG_CK(cudaGetLastError());
        MCG_CK(cudaMemcpyAsync(h_W.data(), d_W, sizeof(double) * nimg_tot * Tmax, cudaMemcpyDeviceToHost, st));
        MCG_CK(cudaStreamSynchronize(st));
        // mean over the images of each vector, in image order
        size_t q0 = 0;
        for (int v = 0; v < nvec; ++v) {
            const size_t ni = imgs[v].size();
            for (int T_ = 0; T_ < Tmax; ++T_) {
                double acc = 0.0;
                for (size_t k = 0; k < ni; ++k) acc += h_W[(q0 + k) * Tmax + T_];
                W_host[((size_t)f * nvec + v) * Tmax + T_] = acc / (double)ni;
            }
            q0 += ni;
        }
    }
    note_launches(launches);
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

int compute_wilson_loops_offaxis(const void* U, int prec, const Geom& g, int nfields, const int* vecs, int nvec,
                                 int Tmax, double* W_host, cudaStream_t st) {
    if (prec == MCG_F64)
        return wilson_offaxis_impl<double>((const cplx<double>*)U, g, nfields, vecs, nvec, Tmax, W_host, st);
    return wilson_offaxis_impl<float>((const cplx<float>*)U, g, nfields, vecs, nvec, Tmax, W_host, st);
}

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_observables)

}  // namespace mcg
