// Field-level kernels: layout conversion, gauge transforms, re-unitarisation,
// plaquette, the MCG functional, Z3 center projection and P-vortex counting.
// All are HBM-bound streaming kernels (one thread per site of one parity).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "mcg_common.cuh"
#include "mcg_internal.h"

namespace mcg {

constexpr int FT = 256;  // threads per block for the streaming kernels

static inline int blocks_for(long long n, int nt) { return (int)((n + nt - 1) / nt); }

// ---------------------------------------------------------------------------
// canonical <-> SoA
// ---------------------------------------------------------------------------
// thread per (field, site lexicographic i); canonical complex128 U[i][mu][e]
template <typename T>
__global__ void k_pack_links(const double2* __restrict__ canon, cplx<T>* __restrict__ U, Geom g, int nfields) {
    const long long V = 2LL * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nfields) return;
    const int f = (int)(id / V);
    const int i = (int)(id - (long long)f * V);
    int c[4];
    int r = i;
    c[0] = r % g.n[0];
    r /= g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1, s = i >> 1;
    const double2* src = canon + ((size_t)f * V + i) * 36;
    cplx<T>* dst = U + (size_t)f * link_elems(g);
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const double2 v = src[mu * 9 + e];
            dst[lidx(g, mu, p, e, s)] = mk((T)v.x, (T)v.y);
        }
}

template <typename T>
__global__ void k_unpack_links(const cplx<T>* __restrict__ U, double2* __restrict__ canon, Geom g, int nfields) {
    const long long V = 2LL * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nfields) return;
    const int f = (int)(id / V);
    const int i = (int)(id - (long long)f * V);
    int c[4];
    int r = i;
    c[0] = r % g.n[0];
    r /= g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1, s = i >> 1;
    double2* dst = canon + ((size_t)f * V + i) * 36;
    const cplx<T>* src = U + (size_t)f * link_elems(g);
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const cplx<T> v = src[lidx(g, mu, p, e, s)];
            dst[mu * 9 + e] = make_double2((double)v.x, (double)v.y);
        }
}

template <typename T>
__global__ void k_pack_gauge(const double2* __restrict__ canon, cplx<T>* __restrict__ G, Geom g, int nfields,
                             int unpack) {
    const long long V = 2LL * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nfields) return;
    const int f = (int)(id / V);
    const int i = (int)(id - (long long)f * V);
    int c[4];
    int r = i;
    c[0] = r % g.n[0];
    r /= g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1, s = i >> 1;
    double2* cn = const_cast<double2*>(canon) + ((size_t)f * V + i) * 9;
    cplx<T>* so = G + (size_t)f * gauge_elems(g);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        if (unpack) {
            const cplx<T> v = so[gidx(g, p, e, s)];
            cn[e] = make_double2((double)v.x, (double)v.y);
        } else {
            const double2 v = cn[e];
            so[gidx(g, p, e, s)] = mk((T)v.x, (T)v.y);
        }
    }
}

__global__ void k_unpack_center(const int8_t* __restrict__ Z, int8_t* __restrict__ canon, Geom g, int nfields) {
    const long long V = 2LL * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nfields) return;
    const int f = (int)(id / V);
    const int i = (int)(id - (long long)f * V);
    int c[4];
    int r = i;
    c[0] = r % g.n[0];
    r /= g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1, s = i >> 1;
    for (int mu = 0; mu < 4; ++mu) canon[((size_t)f * V + i) * 4 + mu] = Z[(size_t)f * 8 * g.vh + (size_t)(mu * 2 + p) * g.vh + s];
}

template <typename TS, typename TD>
__global__ void k_convert(const cplx<TS>* __restrict__ src, cplx<TD>* __restrict__ dst, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const cplx<TS> v = src[k];
        dst[k] = mk((TD)v.x, (TD)v.y);
    }
}

template <typename T>
__global__ void k_identity_gauge(cplx<T>* __restrict__ G, Geom g, int nfields) {
    const long long n = (long long)g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / g.vh), s = (int)(id - (long long)f * g.vh);
    cplx<T>* Gf = G + (size_t)f * gauge_elems(g);
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int e = 0; e < 9; ++e) Gf[gidx(g, p, e, s)] = mk((T)((e % 4) == 0 ? 1 : 0), (T)0);
}

// ---------------------------------------------------------------------------
// gauge transform, in place: U_mu(x) <- Omega(x) U_mu(x) Omega(x+mu)^dag
// thread per (field, parity, site)
// ---------------------------------------------------------------------------
template <typename TU, typename TG>
__device__ __forceinline__ void apply_site(cplx<TU>* __restrict__ U, const cplx<TG>* __restrict__ G, const Geom& g,
                                           int p, int s) {
    int c[4];
    eo_coords(g, p, s, c);
    cplx<double> Om[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const cplx<TG> v = G[gidx(g, p, e, s)];
        Om[e] = mk((double)v.x, (double)v.y);
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int sf = eo_neighbor(g, c, mu, +1);
        cplx<double> u[9], on[9], t[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const cplx<TU> v = U[lidx(g, mu, p, e, s)];
            u[e] = mk((double)v.x, (double)v.y);
            const cplx<TG> w = G[gidx(g, p ^ 1, e, sf)];
            on[e] = mk((double)w.x, (double)w.y);
        }
        m3_mul(Om, u, t);
        m3_mul_nd(t, on, u);
#pragma unroll
        for (int e = 0; e < 9; ++e) U[lidx(g, mu, p, e, s)] = mk((TU)u[e].x, (TU)u[e].y);
    }
}

template <typename T>
__global__ void __launch_bounds__(FT) k_apply_gauge(cplx<T>* __restrict__ U, const cplx<T>* __restrict__ G, Geom g,
                                                     int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    apply_site<T, T>(U + (size_t)f * link_elems(g), G + (size_t)f * gauge_elems(g), g, p, s);
}

template <typename T>
__global__ void __launch_bounds__(FT) k_reunit_all(cplx<T>* __restrict__ M, int per_site, Geom g, int nfields) {
    // per_site = 4 (links) or 1 (gauge): matrices of one site-parity slot
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    cplx<T>* Mf = M + (size_t)f * (per_site == 4 ? link_elems(g) : gauge_elems(g));
    for (int mu = 0; mu < per_site; ++mu) {
        cplx<T> m[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = Mf[((size_t)((mu * 2 + p) * 9 + e)) * g.vh + s];
        m3_reunitarise(m);
#pragma unroll
        for (int e = 0; e < 9; ++e) Mf[((size_t)((mu * 2 + p) * 9 + e)) * g.vh + s] = m[e];
    }
}

// Mixed-precision hand-off, pass 1: W64 = reunit(W) written to scratch (W in
// the compact FP32 form: rows 0 and 1; the FP64 re-unitarisation rebuilds row
// 2 from them), G64 <- reunit(W64 G64).
__global__ void __launch_bounds__(FT) k_handoff_gauge(const float4* __restrict__ W, const float4* __restrict__ Wlo,
                                                      cplx<double>* __restrict__ W64, cplx<double>* __restrict__ G,
                                                      Geom g, int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    const size_t off = (size_t)f * gauge_elems(g);
    const float4* Wf = W + (size_t)f * c12_gauge_chunks(g);
    cplx<double> w[9], o[9], t[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 v = Wf[c12_gidx(g, p, q, s)];
        w[2 * q] = mk((double)v.x, (double)v.y);
        w[2 * q + 1] = mk((double)v.z, (double)v.w);
        if (Wlo) {
            const float4 l = Wlo[(size_t)f * c12_gauge_chunks(g) + c12_gidx(g, p, q, s)];
            w[2 * q] = mk(w[2 * q].x + (double)l.x, w[2 * q].y + (double)l.y);
            w[2 * q + 1] = mk(w[2 * q + 1].x + (double)l.z, w[2 * q + 1].y + (double)l.w);
        }
    }
#pragma unroll
    for (int e = 6; e < 9; ++e) w[e] = mk(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < 9; ++e) o[e] = G[off + gidx(g, p, e, s)];
    m3_reunitarise(w);
    m3_mul(w, o, t);
    m3_reunitarise(t);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        W64[off + gidx(g, p, e, s)] = w[e];
        G[off + gidx(g, p, e, s)] = t[e];
    }
}

// Full layout (FP64 or FP32) -> compact FP32 working storage, for `nmat`
// matrices per site and parity (4: links, 1: gauge transform): rows 0 and 1
// rounded to FP32.
template <typename TS>
__global__ void __launch_bounds__(FT) k_to_c12(const cplx<TS>* __restrict__ src, float4* __restrict__ dst, Geom g,
                                               int nmat, int nfields) {
    const long long per_field = 2LL * nmat * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= per_field * nfields) return;
    const int f = (int)(id / per_field);
    const int r = (int)(id - (long long)f * per_field);
    const int mp = r / g.vh, s = r - mp * g.vh;  // mp = matrix * 2 + parity
    const cplx<TS>* sf = src + (size_t)f * 18 * nmat * g.vh + (size_t)mp * 9 * g.vh + s;
    float4* df = dst + (size_t)f * 6 * nmat * g.vh + (size_t)mp * 3 * g.vh + s;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const cplx<TS> a = sf[(size_t)(2 * q) * g.vh], b = sf[(size_t)(2 * q + 1) * g.vh];
        df[(size_t)q * g.vh] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

// Compact FP32 -> full FP32 layout, row 2 rebuilt as conj(row0 x row1).
__global__ void __launch_bounds__(FT) k_from_c12(const float4* __restrict__ src, cplx<float>* __restrict__ dst,
                                                 Geom g, int nmat, int nfields) {
    const long long per_field = 2LL * nmat * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= per_field * nfields) return;
    const int f = (int)(id / per_field);
    const int r = (int)(id - (long long)f * per_field);
    const int mp = r / g.vh, s = r - mp * g.vh;
    const float4* sf = src + (size_t)f * 6 * nmat * g.vh + (size_t)mp * 3 * g.vh + s;
    cplx<float>* df = dst + (size_t)f * 18 * nmat * g.vh + (size_t)mp * 9 * g.vh + s;
    cplx<float> m[6];
    c12_load(sf, (size_t)g.vh, m);
#pragma unroll
    for (int e = 0; e < 6; ++e) df[(size_t)e * g.vh] = m[e];
#pragma unroll
    for (int k = 0; k < 3; ++k) df[(size_t)(6 + k) * g.vh] = row2_entry(m, k);
}

__global__ void __launch_bounds__(FT) k_identity_c12(float4* __restrict__ W, Geom g, int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    float4* Wf = W + (size_t)f * c12_gauge_chunks(g);
    Wf[c12_gidx(g, p, 0, s)] = make_float4(1.f, 0.f, 0.f, 0.f);  // (W00, W01)
    Wf[c12_gidx(g, p, 1, s)] = make_float4(0.f, 0.f, 0.f, 0.f);  // (W02, W10)
    Wf[c12_gidx(g, p, 2, s)] = make_float4(1.f, 0.f, 0.f, 0.f);  // (W11, W12)
}

// ---------------------------------------------------------------------------
// plaquette and functional: per-field sums via per-block partials
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FT) k_plaquette(const cplx<T>* __restrict__ U, Geom g, int bpf,
                                                  double* __restrict__ partial) {
    const int f = blockIdx.x / bpf;
    const int s2 = (blockIdx.x - f * bpf) * FT + threadIdx.x;  // 0 .. 2*vh-1
    const cplx<T>* Uf = U + (size_t)f * link_elems(g);
    double acc = 0.0;
    if (s2 < 2 * g.vh) {
        const int p = s2 / g.vh, s = s2 - p * g.vh;
        int c[4];
        eo_coords(g, p, s, c);
        for (int mu = 0; mu < 4; ++mu) {
            const int smu = eo_neighbor(g, c, mu, +1);
            cplx<double> a[9], t[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                const cplx<T> v = Uf[lidx(g, mu, p, e, s)];
                a[e] = mk((double)v.x, (double)v.y);
            }
            for (int nu = mu + 1; nu < 4; ++nu) {
                const int snu = eo_neighbor(g, c, nu, +1);
                cplx<double> b[9], m[9], q[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    const cplx<T> v = Uf[lidx(g, nu, p ^ 1, e, smu)];
                    b[e] = mk((double)v.x, (double)v.y);
                }
                m3_mul(a, b, t);  // U_mu(x) U_nu(x+mu)
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    const cplx<T> v = Uf[lidx(g, mu, p ^ 1, e, snu)];
                    m[e] = mk((double)v.x, (double)v.y);
                }
                m3_mul_nd(t, m, q);  // ... U_mu(x+nu)^dag
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    const cplx<T> v = Uf[lidx(g, nu, p, e, s)];
                    m[e] = mk((double)v.x, (double)v.y);
                }
                // Re tr(q m^dag) = sum_ij Re(q_ij conj(m_ij))
                double tr = 0.0;
#pragma unroll
                for (int e = 0; e < 9; ++e) tr += q[e].x * m[e].x + q[e].y * m[e].y;
                acc += tr / 3.0;
            }
        }
    }
    __shared__ double red[FT / 32];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(FT) k_functional_all(const cplx<T>* __restrict__ U, Geom g, int bpf,
                                                       double* __restrict__ partial) {
    const int f = blockIdx.x / bpf;
    const int s2 = (blockIdx.x - f * bpf) * FT + threadIdx.x;
    const cplx<T>* Uf = U + (size_t)f * link_elems(g);
    double acc = 0.0;
    if (s2 < 2 * g.vh) {
        const int p = s2 / g.vh, s = s2 - p * g.vh;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const cplx<T> a = Uf[lidx(g, mu, p, 0, s)], b = Uf[lidx(g, mu, p, 4, s)], c = Uf[lidx(g, mu, p, 8, s)];
            const double tr = (double)(a.x + b.x + c.x), ti = (double)(a.y + b.y + c.y);
            acc += tr * tr + ti * ti;
        }
    }
    __shared__ double red[FT / 32];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int bpf, double* __restrict__ out) {
    const int f = blockIdx.x;
    double v = 0.0;
    for (int k = threadIdx.x; k < bpf; k += blockDim.x) v += partial[(size_t)f * bpf + k];
    __shared__ double red[8];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) out[f] = tot;
}

// ---------------------------------------------------------------------------
// center projection (decision in FP64, exact comparisons) and vortex counting
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(FT) k_center_project(const cplx<T>* __restrict__ U, int8_t* __restrict__ Z, Geom g,
                                                       int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    const cplx<T>* Uf = U + (size_t)f * link_elems(g);
    int8_t* Zf = Z + (size_t)f * 8 * g.vh;
    const double sqrt3 = 1.7320508075688772;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const cplx<T> a = Uf[lidx(g, mu, p, 0, s)], b = Uf[lidx(g, mu, p, 4, s)], c = Uf[lidx(g, mu, p, 8, s)];
        const double re = __dadd_rn(__dadd_rn((double)a.x, (double)b.x), (double)c.x);
        const double im = __dadd_rn(__dadd_rn((double)a.y, (double)b.y), (double)c.y);
        const double lim = __dmul_rn(sqrt3, re);
        int8_t m;
        if (re >= 0.0 && fabs(im) <= lim)
            m = 0;
        else if (im >= 0.0)
            m = 1;
        else
            m = -1;
        Zf[(size_t)(mu * 2 + p) * g.vh + s] = m;
    }
}

// per (field, parity, site): 6 plaquettes; counts[f*7 + 1 + plane]
__global__ void __launch_bounds__(FT) k_vortex_count(const int8_t* __restrict__ Z, Geom g, int nfields,
                                                     unsigned long long* __restrict__ counts) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int cnt[6] = {0, 0, 0, 0, 0, 0};
    int f = 0;
    if (id < n) {
        f = (int)(id / (2LL * g.vh));
        const int r = (int)(id - (long long)f * 2 * g.vh);
        const int p = r / g.vh, s = r - p * g.vh;
        const int8_t* Zf = Z + (size_t)f * 8 * g.vh;
        int c[4];
        eo_coords(g, p, s, c);
        int pl = 0;
        for (int mu = 0; mu < 4; ++mu) {
            const int smu = eo_neighbor(g, c, mu, +1);
            for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
                const int snu = eo_neighbor(g, c, nu, +1);
                const int v = Zf[(size_t)(mu * 2 + p) * g.vh + s] + Zf[(size_t)(nu * 2 + (p ^ 1)) * g.vh + smu] -
                              Zf[(size_t)(mu * 2 + (p ^ 1)) * g.vh + snu] - Zf[(size_t)(nu * 2 + p) * g.vh + s];
                cnt[pl] = (((v % 3) + 3) % 3) != 0;
            }
        }
    }
    // a block may straddle two fields only at field boundaries: reduce per warp
    // on the warp's first field and fall back to per-thread atomics otherwise
    const int f0 = __shfl_sync(0xffffffffu, f, 0);
    const bool uniform = __all_sync(0xffffffffu, f == f0 || id >= n);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (uniform) {
            const int w = __reduce_add_sync(0xffffffffu, cnt[k]);
            if ((threadIdx.x & 31) == 0 && w) atomicAdd(&counts[(size_t)f0 * 7 + 1 + k], (unsigned long long)w);
        } else if (cnt[k]) {
            atomicAdd(&counts[(size_t)f * 7 + 1 + k], 1ULL);
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int launch_convert(const void* src, int sp, void* dst, int dp, size_t n, cudaStream_t st) {
    const int nb = (int)std::min<size_t>((n + FT - 1) / FT, 152 * 64);
    if (n == 0) return 0;
    if (sp == MCG_F64 && dp == MCG_F32)
        k_convert<double, float><<<nb, FT, 0, st>>>((const cplx<double>*)src, (cplx<float>*)dst, n);
    else if (sp == MCG_F32 && dp == MCG_F64)
        k_convert<float, double><<<nb, FT, 0, st>>>((const cplx<float>*)src, (cplx<double>*)dst, n);
    else if (sp == MCG_F64)
        k_convert<double, double><<<nb, FT, 0, st>>>((const cplx<double>*)src, (cplx<double>*)dst, n);
    else
        k_convert<float, float><<<nb, FT, 0, st>>>((const cplx<float>*)src, (cplx<float>*)dst, n);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_pack(const double* canon, void* soa, int prec, const Geom& g, int nfields, int what, int unpack,
                cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    const int nb = blocks_for(n, FT);
    if (what == 0) {
        if (!unpack) {
            if (prec == MCG_F64)
                k_pack_links<double><<<nb, FT, 0, st>>>((const double2*)canon, (cplx<double>*)soa, g, nfields);
            else
                k_pack_links<float><<<nb, FT, 0, st>>>((const double2*)canon, (cplx<float>*)soa, g, nfields);
        } else {
            if (prec == MCG_F64)
                k_unpack_links<double><<<nb, FT, 0, st>>>((const cplx<double>*)soa, (double2*)canon, g, nfields);
            else
                k_unpack_links<float><<<nb, FT, 0, st>>>((const cplx<float>*)soa, (double2*)canon, g, nfields);
        }
    } else {
        if (prec == MCG_F64)
            k_pack_gauge<double><<<nb, FT, 0, st>>>((const double2*)canon, (cplx<double>*)soa, g, nfields, unpack);
        else
            k_pack_gauge<float><<<nb, FT, 0, st>>>((const double2*)canon, (cplx<float>*)soa, g, nfields, unpack);
    }
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_unpack_center(const int8_t* Z, int8_t* canon, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    k_unpack_center<<<blocks_for(n, FT), FT, 0, st>>>(Z, canon, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

// ---------------------------------------------------------------------------
// Input validation: every matrix finite and in SU(3) to within tol
// ---------------------------------------------------------------------------
// Matrix m of a field (nslots x Vh matrices: 8 = 4 directions x 2 parities
// for links, 2 parities for a gauge transform) has entry e at
// ((m / Vh) * 9 + e) * Vh + m % Vh.  A matrix fails if an entry is not finite,
// if max_ij |(M M^dag - 1)_ij| > tol or if |det M - 1| > tol (FP32 arithmetic:
// its rounding, ~1e-7, is far below the tolerances used).  bad[0]: number of
// failing matrices; bad[1]: smallest failing global matrix index.
template <typename T>
__global__ void k_check_su3(const cplx<T>* __restrict__ M, int nslots, size_t vh, size_t nmat, float tol,
                            bool finite_only, unsigned long long* __restrict__ bad) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmat) return;
    const size_t per_field = (size_t)nslots * vh;
    const size_t f = i / per_field, m = i % per_field;
    const cplx<T>* base = M + f * per_field * 9 + (m / vh) * 9 * vh + m % vh;
    cplx<float> a[9];
    bool finite = true;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const cplx<T> v = base[(size_t)e * vh];
        finite = finite && isfinite(v.x) && isfinite(v.y);
        a[e] = mk((float)v.x, (float)v.y);
    }
    bool ok = finite;
    if (ok && !finite_only) {
        float dev = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = r; c < 3; ++c) {
                cplx<float> d = mk(r == c ? -1.f : 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < 3; ++k) d = cfmac(a[3 * r + k], a[3 * c + k], d);
                dev = fmaxf(dev, fmaxf(fabsf(d.x), fabsf(d.y)));
            }
        // det by the first row's cofactors
        const cplx<float> c0 = csub(cmul(a[4], a[8]), cmul(a[5], a[7]));
        const cplx<float> c1 = csub(cmul(a[5], a[6]), cmul(a[3], a[8]));
        const cplx<float> c2 = csub(cmul(a[3], a[7]), cmul(a[4], a[6]));
        const cplx<float> det = cadd(cadd(cmul(a[0], c0), cmul(a[1], c1)), cmul(a[2], c2));
        dev = fmaxf(dev, fmaxf(fabsf(det.x - 1.f), fabsf(det.y)));
        ok = dev <= tol;  // false for NaN too
    }
    if (!ok) {
        atomicAdd(&bad[0], 1ull);
        atomicMin(&bad[1], (unsigned long long)i);
    }
}

int validate_su3(const void* M, int prec, const Geom& g, int nslots, int nfields, const char* what,
                 cudaStream_t st, bool finite_only) {
    int rc = 0;
    unsigned long long* d_bad = (unsigned long long*)scratch_device("check.bad", 2 * sizeof(unsigned long long), &rc);
    if (rc) return rc;
    unsigned long long* h_bad = (unsigned long long*)scratch_host("check.bad", 2 * sizeof(unsigned long long), &rc);
    if (rc) return rc;
    MCG_CK(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st));
    MCG_CK(cudaMemsetAsync(d_bad + 1, 0xff, sizeof(unsigned long long), st));
    const size_t vh = (size_t)g.vh, nmat = (size_t)nslots * vh * nfields;
    const unsigned nb = (unsigned)((nmat + FT - 1) / FT);
    if (prec == MCG_F64)
        k_check_su3<double><<<nb, FT, 0, st>>>((const cplx<double>*)M, nslots, vh, nmat, kSU3TolF64, finite_only,
                                               d_bad);
    else
        k_check_su3<float><<<nb, FT, 0, st>>>((const cplx<float>*)M, nslots, vh, nmat, kSU3TolF32, finite_only,
                                              d_bad);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    MCG_CK(cudaMemcpyAsync(h_bad, d_bad, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MCG_CK(cudaStreamSynchronize(st));
    if (h_bad[0] == 0) return 0;
    const size_t i = (size_t)h_bad[1], per_field = (size_t)nslots * vh;
    const size_t f = i / per_field, slot = (i % per_field) / vh, s = i % vh;
    char buf[320];
    if (finite_only)
        snprintf(buf, sizeof buf, "%s: %llu matrices have non-finite entries (first: field %zu, mu %zu, parity %zu, "
                 "in-parity site %zu)", what, h_bad[0], f, slot / 2, slot % 2, s);
    else if (nslots == 8)
        snprintf(buf, sizeof buf,
                 "%s: %llu matrices are not finite or not in SU(3) to %g (first: field %zu, mu %zu, parity %zu, "
                 "in-parity site %zu)",
                 what, h_bad[0], prec == MCG_F64 ? kSU3TolF64 : kSU3TolF32, f, slot / 2, slot % 2, s);
    else
        snprintf(buf, sizeof buf,
                 "%s: %llu matrices are not finite or not in SU(3) to %g (first: field %zu, parity %zu, "
                 "in-parity site %zu)",
                 what, h_bad[0], prec == MCG_F64 ? kSU3TolF64 : kSU3TolF32, f, slot, s);
    return fail(MCG_BAD_INPUT, buf);
}

// ---------------------------------------------------------------------------
// Arithmetic throughput probes (instrumentation): FMA rate of the FP64 pipe,
// the FP32 pipe and the packed FP32 instruction (two FMAs on a register pair)
// ---------------------------------------------------------------------------
// Each thread runs kChains independent FMA chains x <- x * m + a for `iters`
// iterations (no dependency between chains, so the pipes, not the latency,
// bound the rate); the result is stored only if it equals an impossible value,
// which keeps the work without memory traffic.
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(1.0 + 1e-3 * c + 1e-7 * threadIdx.x);
    const T m = (T)0.999999, a = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], m, a);
    }
    T sum = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) sum += x[c];
    if (sum == (T)-1.25) out[threadIdx.x] = sum;
}

__global__ void __launch_bounds__(256) k_fma2_probe(float* out, int iters) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(1.f + 1e-3f * c, 1.f + 1e-7f * threadIdx.x);
    const float2 m = make_float2(0.999999f, 0.999999f), a = make_float2(1e-7f, 1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], m, a);
    }
    float sum = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) sum += x[c].x + x[c].y;
    if (sum == -1.25f) out[threadIdx.x] = sum;
}

int probe_peaks(double* tflops, cudaStream_t st) {
    int dev = 0, nsm = 0, rc = 0;
    MCG_CK(cudaGetDevice(&dev));
    MCG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    double* sink = (double*)scratch_device("probe.sink", 256 * sizeof(double), &rc);
    if (rc) return rc;
    const unsigned blocks = (unsigned)nsm * 8;
    const double threads = (double)blocks * 256;
    cudaEvent_t e0, e1;
    MCG_CK(cudaEventCreate(&e0));
    MCG_CK(cudaEventCreate(&e1));
    for (int kind = 0; kind < 3; ++kind) {
        // iterations for ~20 ms, from a short calibration launch
        int iters = 64;
        float ms = 0.f;
        for (int pass = 0; pass < 2; ++pass) {
            cudaEventRecord(e0, st);
            if (kind == 0)
                k_fma_probe<double><<<blocks, 256, 0, st>>>(sink, iters);
            else if (kind == 1)
                k_fma_probe<float><<<blocks, 256, 0, st>>>((float*)sink, iters);
            else
                k_fma2_probe<<<blocks, 256, 0, st>>>((float*)sink, iters);
            cudaEventRecord(e1, st);
            MCG_CK(cudaEventSynchronize(e1));
            MCG_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (pass == 0) iters = (int)std::min(1.0e7, std::max(64.0, iters * 20.0 / std::max(ms, 1e-3f)));
        }
        const double flop_per_iter = threads * kChains * 2.0 * (kind == 2 ? 2.0 : 1.0);
        tflops[kind] = flop_per_iter * iters / (ms * 1e-3) / 1e12;
    }
    note_launches(6);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MCG_CK(cudaGetLastError());
    return 0;
}

int launch_identity_gauge(void* G, int prec, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = (long long)g.vh * nfields;
    if (prec == MCG_F64)
        k_identity_gauge<double><<<blocks_for(n, FT), FT, 0, st>>>((cplx<double>*)G, g, nfields);
    else
        k_identity_gauge<float><<<blocks_for(n, FT), FT, 0, st>>>((cplx<float>*)G, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_apply_gauge(void* U, const void* G, int prec, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    if (prec == MCG_F64)
        k_apply_gauge<double><<<blocks_for(n, FT), FT, 0, st>>>((cplx<double>*)U, (const cplx<double>*)G, g, nfields);
    else
        k_apply_gauge<float><<<blocks_for(n, FT), FT, 0, st>>>((cplx<float>*)U, (const cplx<float>*)G, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_reunitarise(void* M, int which, int prec, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    const int per = which == 0 ? 4 : 1;
    if (prec == MCG_F64)
        k_reunit_all<double><<<blocks_for(n, FT), FT, 0, st>>>((cplx<double>*)M, per, g, nfields);
    else
        k_reunit_all<float><<<blocks_for(n, FT), FT, 0, st>>>((cplx<float>*)M, per, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

static int reduce_per_field(int which, const void* U, int prec, const Geom& g, int nfields, double* out_host,
                            cudaStream_t st) {
    const int bpf = blocks_for(2LL * g.vh, FT);
    int rc = 0;
    double* partial = (double*)scratch_device("obs.partial", sizeof(double) * (size_t)bpf * nfields, &rc);
    if (rc) return rc;
    double* d_out = (double*)scratch_device("obs.out", sizeof(double) * nfields, &rc);
    if (rc) return rc;
    const int nb = bpf * nfields;
    if (which == 0) {
        if (prec == MCG_F64)
            k_plaquette<double><<<nb, FT, 0, st>>>((const cplx<double>*)U, g, bpf, partial);
        else
            k_plaquette<float><<<nb, FT, 0, st>>>((const cplx<float>*)U, g, bpf, partial);
    } else {
        if (prec == MCG_F64)
            k_functional_all<double><<<nb, FT, 0, st>>>((const cplx<double>*)U, g, bpf, partial);
        else
            k_functional_all<float><<<nb, FT, 0, st>>>((const cplx<float>*)U, g, bpf, partial);
    }
    k_sum_partials<<<nfields, 256, 0, st>>>(partial, bpf, d_out);
    MCG_CK(cudaGetLastError());
    note_launches(2);
    MCG_CK(cudaMemcpyAsync(out_host, d_out, sizeof(double) * nfields, cudaMemcpyDeviceToHost, st));
    MCG_CK(cudaStreamSynchronize(st));
    if (which == 0)
        for (int f = 0; f < nfields; ++f) out_host[f] /= 6.0 * 2.0 * g.vh;
    return 0;
}

int compute_plaquette(const void* U, int prec, const Geom& g, int nfields, double* out_host, cudaStream_t st) {
    return reduce_per_field(0, U, prec, g, nfields, out_host, st);
}

int compute_functional(const void* U, int prec, const Geom& g, int nfields, double* out_host, cudaStream_t st) {
    return reduce_per_field(1, U, prec, g, nfields, out_host, st);
}

int compute_center(const void* U, int prec, int8_t* Z, const Geom& g, int nfields, long long* counts_host,
                   cudaStream_t st) {
    int rc = 0;
    unsigned long long* d_counts =
        (unsigned long long*)scratch_device("center.counts", sizeof(unsigned long long) * 7 * nfields, &rc);
    if (rc) return rc;
    const long long n = 2LL * g.vh * nfields;
    if (prec == MCG_F64)
        k_center_project<double><<<blocks_for(n, FT), FT, 0, st>>>((const cplx<double>*)U, Z, g, nfields);
    else
        k_center_project<float><<<blocks_for(n, FT), FT, 0, st>>>((const cplx<float>*)U, Z, g, nfields);
    MCG_CK(cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * 7 * nfields, st));
    k_vortex_count<<<blocks_for(n, FT), FT, 0, st>>>(Z, g, nfields, d_counts);
    MCG_CK(cudaGetLastError());
    note_launches(2);
    if (counts_host) {
        MCG_CK(cudaMemcpyAsync(counts_host, d_counts, sizeof(long long) * 7 * nfields, cudaMemcpyDeviceToHost, st));
        MCG_CK(cudaStreamSynchronize(st));
        for (int f = 0; f < nfields; ++f) {
            long long t = 0;
            for (int k = 1; k < 7; ++k) t += counts_host[f * 7 + k];
            counts_host[f * 7] = t;
        }
    }
    return 0;
}

int launch_handoff(const void* W32, const void* W32lo, double* U64, double* G64, const Geom& g, int nfields,
                   cudaStream_t st) {
    int rc = 0;
    cplx<double>* W64 =
        (cplx<double>*)scratch_device("handoff.W64", sizeof(cplx<double>) * gauge_elems(g) * nfields, &rc);
    if (rc) return rc;
    const long long n = 2LL * g.vh * nfields;
    k_handoff_gauge<<<blocks_for(n, FT), FT, 0, st>>>((const float4*)W32, (const float4*)W32lo, W64,
                                                      (cplx<double>*)G64, g, nfields);
    k_apply_gauge<double><<<blocks_for(n, FT), FT, 0, st>>>((cplx<double>*)U64, W64, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(2);
    return 0;
}

int launch_to_c12(const void* src, int src_prec, void* dst, const Geom& g, int nmat, int nfields, cudaStream_t st) {
    const long long n = 2LL * nmat * g.vh * nfields;
    if (src_prec == MCG_F64)
        k_to_c12<double><<<blocks_for(n, FT), FT, 0, st>>>((const cplx<double>*)src, (float4*)dst, g, nmat, nfields);
    else
        k_to_c12<float><<<blocks_for(n, FT), FT, 0, st>>>((const cplx<float>*)src, (float4*)dst, g, nmat, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_from_c12(const void* src, void* dst, const Geom& g, int nmat, int nfields, cudaStream_t st) {
    const long long n = 2LL * nmat * g.vh * nfields;
    k_from_c12<<<blocks_for(n, FT), FT, 0, st>>>((const float4*)src, (cplx<float>*)dst, g, nmat, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_identity_c12(void* W, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    k_identity_c12<<<blocks_for(n, FT), FT, 0, st>>>((float4*)W, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

}  // namespace mcg

// ---------------------------------------------------------------------------
// Plaquette without any allocation (mcg_plaquette_static)
// ---------------------------------------------------------------------------
namespace mcg {
// sum of one field's block partials in a fixed order, scaled, to out[f]
__global__ void k_static_finish(const double* __restrict__ partial, int bpf, double scale, double* __restrict__ out) {
    const int f = blockIdx.x;
    double v = 0.0;
    for (int k = threadIdx.x; k < bpf; k += blockDim.x) v += partial[(size_t)f * bpf + k];
    __shared__ double red[8];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) out[f] = tot * scale;
}
}  // namespace mcg

// Some callers cannot let a library call cudaMalloc: an application whose
// device memory is fully handed to its own pool allocator (a new cudaMalloc
// would fail or break its accounting), a latency-critical loop that cannot
// absorb the device-wide synchronisation cudaFree implies, or code that
// must keep its memory footprint fixed after start-up.  For them this entry
// point keeps its only scratch, the per-block partial sums, in a fixed array
// compiled into the library; the caller passes the field and a device buffer
// for the result.  Every GPU that loads the library holds this array until
// the process exits.
namespace mcg {

constexpr int kStaticPartials = 1 << 16;  // 65 536 doubles = 512 KiB
static __device__ __align__(256) double g_static_partials[kStaticPartials];

static std::mutex g_static_mu;
static double* g_static_addr[64];  // symbol address per device, resolved once

// Resolve the device address of the static partials for the current device.
static int static_partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(MCG_BAD_ARG, "device index beyond 63");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static partials)");
        g_static_addr[dev] = (double*)p;
    }
    *out = g_static_addr[dev];
    return 0;
}

void static_release() {
    std::lock_guard<std::mutex> lk(g_static_mu);
    for (auto& p : g_static_addr) p = nullptr;
}

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_field)

}  // namespace mcg

extern "C" int mcg_plaquette_static(const void* U, double* out, const mcg_lattice* lat, cudaStream_t stream) {
    using namespace mcg;
    Geom g;
    int rc = check_lattice(lat, &g);
    if (rc) return rc;
    if (!U || !out) return fail(MCG_BAD_ARG, "null pointer");
    const long long V = 2LL * g.vh;
    const long long bpf = (V + FT - 1) / FT;
    if (bpf * lat->nfields > kStaticPartials)
        return fail(MCG_BAD_ARG, "mcg_plaquette_static: nfields * ceil(V / 256) exceeds the 65536 static partial "
                                 "sums (at most 16 777 216 sites in total); use mcg_plaquette");
    double* partial = nullptr;
    if ((rc = static_partials_address(&partial))) return rc;
    // every partial slot read below is written by its block first: nothing in
    // the shared array has to start at zero
    const int nb = (int)bpf * lat->nfields;
    if (lat->precision == MCG_F64)
        k_plaquette<double><<<nb, FT, 0, stream>>>((const cplx<double>*)U, g, (int)bpf, partial);
    else
        k_plaquette<float><<<nb, FT, 0, stream>>>((const cplx<float>*)U, g, (int)bpf, partial);
    k_static_finish<<<lat->nfields, 256, 0, stream>>>(partial, (int)bpf, 1.0 / (6.0 * (double)V), out);
    MCG_CK(cudaGetLastError());
    note_launches(2);
    return MCG_OK;
}
