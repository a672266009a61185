// Device-side building blocks shared by the libmcg kernels: complex numbers,
// 3x3 complex matrix helpers, the even/odd SoA field layout and lattice
// geometry.  Everything here is for sm_103a; none of it is used by the CPU
// oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcg.h"

namespace mcg {

// ---------------------------------------------------------------------------
// complex arithmetic (vector-aligned so a link element is one 8/16-byte load)
// ---------------------------------------------------------------------------
template <typename T>
struct alignas(2 * sizeof(T)) cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> mk(T x, T y) {
    cplx<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
    return mk(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) {
    return mk(a.x - b.x, a.y - b.y);
}
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc + a * b
template <typename T>
__device__ __forceinline__ cplx<T> cfma(cplx<T> a, cplx<T> b, cplx<T> acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + a * conj(b)
template <typename T>
__device__ __forceinline__ cplx<T> cfmac(cplx<T> a, cplx<T> b, cplx<T> acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
    return acc;
}
// acc + conj(a) * b
template <typename T>
__device__ __forceinline__ cplx<T> cfmaca(cplx<T> a, cplx<T> b, cplx<T> acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) {
    return mk(a.x * s, a.y * s);
}
template <typename T>
__device__ __forceinline__ T cnorm2(cplx<T> a) {
    return a.x * a.x + a.y * a.y;
}

// ---------------------------------------------------------------------------
// 3x3 complex matrices held in registers, row-major m[3*i + j]
// ---------------------------------------------------------------------------
template <typename T>
struct M3 {
    cplx<T> m[9];
};

template <typename T>
__device__ __forceinline__ void m3_mul(const cplx<T>* a, const cplx<T>* b, cplx<T>* r) {  // r = a b
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cplx<T> s = cmul(a[3 * i], b[j]);
            s = cfma(a[3 * i + 1], b[3 + j], s);
            s = cfma(a[3 * i + 2], b[6 + j], s);
            r[3 * i + j] = s;
        }
}
template <typename T>
__device__ __forceinline__ void m3_mul_nd(const cplx<T>* a, const cplx<T>* b, cplx<T>* r) {  // r = a b^dag
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cplx<T> s = cmulc(a[3 * i], b[3 * j]);
            s = cfmac(a[3 * i + 1], b[3 * j + 1], s);
            s = cfmac(a[3 * i + 2], b[3 * j + 2], s);
            r[3 * i + j] = s;
        }
}
template <typename T>
__device__ __forceinline__ void m3_mul_dn(const cplx<T>* a, const cplx<T>* b, cplx<T>* r) {  // r = a^dag b
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cplx<T> s = mk(a[i].x * b[j].x + a[i].y * b[j].y, a[i].x * b[j].y - a[i].y * b[j].x);
            s = cfmaca(a[3 + i], b[3 + j], s);
            s = cfmaca(a[6 + i], b[6 + j], s);
            r[3 * i + j] = s;
        }
}

// Re-unitarise in place: normalise row 0, orthogonalise and normalise row 1,
// row 2 = conj(row0 x row1).  Arithmetic in double whatever T is.
template <typename T>
__device__ __forceinline__ void m3_reunitarise(cplx<T>* a) {
    double r0x[3], r0y[3], r1x[3], r1y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r0x[k] = (double)a[k].x;
        r0y[k] = (double)a[k].y;
        r1x[k] = (double)a[3 + k].x;
        r1y[k] = (double)a[3 + k].y;
    }
    double n0 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) n0 += r0x[k] * r0x[k] + r0y[k] * r0y[k];
    n0 = rsqrt(n0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r0x[k] *= n0;
        r0y[k] *= n0;
    }
    double px = 0, py = 0;  // conj(r0) . r1
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        px += r0x[k] * r1x[k] + r0y[k] * r1y[k];
        py += r0x[k] * r1y[k] - r0y[k] * r1x[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r1x[k] -= px * r0x[k] - py * r0y[k];
        r1y[k] -= px * r0y[k] + py * r0x[k];
    }
    double n1 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) n1 += r1x[k] * r1x[k] + r1y[k] * r1y[k];
    n1 = rsqrt(n1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r1x[k] *= n1;
        r1y[k] *= n1;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = mk((T)r0x[k], (T)r0y[k]);
        a[3 + k] = mk((T)r1x[k], (T)r1y[k]);
    }
    // row 2 = conj(r0 x r1): (r0_1 r1_2 - r0_2 r1_1)^*, ...
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        double cx = (r0x[i] * r1x[j] - r0y[i] * r1y[j]) - (r0x[j] * r1x[i] - r0y[j] * r1y[i]);
        double cy = (r0x[i] * r1y[j] + r0y[i] * r1x[j]) - (r0x[j] * r1y[i] + r0y[j] * r1x[i]);
        a[6 + k] = mk((T)cx, (T)(-cy));
    }
}

// ---------------------------------------------------------------------------
// Field layout (the C-ABI contract, see include/mcg.h):
//   site s of parity p (in-parity index s = lexicographic index / 2),
//   link U_mu entry e = 3*row+col:  U[((mu*2 + p)*9 + e)*Vh + s]
//   gauge Omega entry e:            G[(p*9 + e)*Vh + s]
//   center sector of U_mu:          Z[(mu*2 + p)*Vh + s]
// ---------------------------------------------------------------------------
struct Geom {
    int n[4];
    int vh;  // V / 2
};

// ---------------------------------------------------------------------------
// Index checks of the MCG_CHECK build (nvcc -DMCG_CHECK): the layout helpers
// below test every component of an index against its range (direction,
// parity, entry or chunk, site, coordinate); a bad one is counted in a
// device counter of the translation unit and the helper returns index 0, so
// the access stays inside the array and no kernel traps.  Each unit's counter
// is read by the host function its MCG_BOUND_READER defines
// (mcg_bounds_violations sums them).  Without MCG_CHECK the checks compile to
// nothing.
// ---------------------------------------------------------------------------
#ifdef MCG_CHECK
static __device__ unsigned long long g_bound_hits;
__device__ __forceinline__ bool mcg_bad(bool bad) {
    if (bad) atomicAdd(&g_bound_hits, 1ULL);
    return bad;
}
#define MCG_BOUND_READER(fn)                                                   \
    unsigned long long fn(bool reset) {                                        \
        unsigned long long v = 0;                                              \
        cudaMemcpyFromSymbol(&v, g_bound_hits, sizeof v);                      \
        if (reset) {                                                           \
            const unsigned long long z = 0;                                    \
            cudaMemcpyToSymbol(g_bound_hits, &z, sizeof z);                    \
        }                                                                      \
        return v;                                                              \
    }
#else
__device__ __forceinline__ bool mcg_bad(bool) { return false; }
#define MCG_BOUND_READER(fn) \
    unsigned long long fn(bool) { return 0; }
#endif

__host__ __device__ __forceinline__ size_t link_elems(const Geom& g) { return (size_t)72 * g.vh; }
__host__ __device__ __forceinline__ size_t gauge_elems(const Geom& g) { return (size_t)18 * g.vh; }

__device__ __forceinline__ size_t lidx(const Geom& g, int mu, int p, int e, int s) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)mu >= 4u || (unsigned)p >= 2u || (unsigned)e >= 9u || (unsigned)s >= (unsigned)g.vh))
        return 0;
#endif
    return ((size_t)((mu * 2 + p) * 9 + e)) * g.vh + s;
}
__device__ __forceinline__ size_t gidx(const Geom& g, int p, int e, int s) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)p >= 2u || (unsigned)e >= 9u || (unsigned)s >= (unsigned)g.vh)) return 0;
#endif
    return ((size_t)(p * 9 + e)) * g.vh + s;
}

// coordinates (x,y,z,t) of site s in parity p
__device__ __forceinline__ void eo_coords(const Geom& g, int p, int s, int c[4]) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)p >= 2u || (unsigned)s >= (unsigned)g.vh)) s = 0;
#endif
    int i2 = 2 * s;
    int x0 = i2 % g.n[0];
    int r = i2 / g.n[0];
    c[1] = r % g.n[1];
    r /= g.n[1];
    c[2] = r % g.n[2];
    c[3] = r / g.n[2];
    c[0] = x0 + ((c[1] + c[2] + c[3] + p) & 1);
}
__device__ __forceinline__ int eo_index(const Geom& g, const int c[4]) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)c[0] >= (unsigned)g.n[0] || (unsigned)c[1] >= (unsigned)g.n[1] ||
                (unsigned)c[2] >= (unsigned)g.n[2] || (unsigned)c[3] >= (unsigned)g.n[3]))
        return 0;
#endif
    return (c[0] + g.n[0] * (c[1] + g.n[1] * (c[2] + g.n[2] * c[3]))) >> 1;
}
// in-parity index of the neighbour c +- mu (step = +1 or -1), periodic
__device__ __forceinline__ int eo_neighbor(const Geom& g, const int c[4], int mu, int step) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    int v = d[mu] + step;
    d[mu] = v < 0 ? v + g.n[mu] : (v >= g.n[mu] ? v - g.n[mu] : v);
    return eo_index(g, d);
}

template <typename T>
__device__ __forceinline__ void load_link(const cplx<T>* __restrict__ U, const Geom& g, int mu, int p, int s,
                                          cplx<T>* m) {
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = U[lidx(g, mu, p, e, s)];
}
template <typename T>
__device__ __forceinline__ void store_link(cplx<T>* __restrict__ U, const Geom& g, int mu, int p, int s,
                                           const cplx<T>* m) {
#pragma unroll
    for (int e = 0; e < 9; ++e) U[lidx(g, mu, p, e, s)] = m[e];
}

// ---------------------------------------------------------------------------
// Compact FP32 working storage (the FP32 sweep phase): rows 0 and 1 of each
// SU(3) matrix, 12 reals; row 2 is implied, row2 = conj(row0 x row1).  A
// matrix is three float4 chunks, chunk q holding entries 2q and 2q+1 of
// (M00 M01 M02 M10 M11 M12):
//   link U_mu, chunk q:  C[((mu*2 + p)*3 + q)*Vh + s]
//   gauge W, chunk q:    C[(p*3 + q)*Vh + s]
// so one chunk of 32 consecutive sites is one 512-byte coalesced access.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t c12_link_chunks(const Geom& g) { return (size_t)24 * g.vh; }
__host__ __device__ __forceinline__ size_t c12_gauge_chunks(const Geom& g) { return (size_t)6 * g.vh; }
__device__ __forceinline__ size_t c12_lidx(const Geom& g, int mu, int p, int q, int s) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)mu >= 4u || (unsigned)p >= 2u || (unsigned)q >= 3u || (unsigned)s >= (unsigned)g.vh))
        return 0;
#endif
    return ((size_t)((mu * 2 + p) * 3 + q)) * g.vh + s;
}
__device__ __forceinline__ size_t c12_gidx(const Geom& g, int p, int q, int s) {
#ifdef MCG_CHECK
    if (mcg_bad((unsigned)p >= 2u || (unsigned)q >= 3u || (unsigned)s >= (unsigned)g.vh)) return 0;
#endif
    return ((size_t)(p * 3 + q)) * g.vh + s;
}

// entry (2, k) of an SU(3) matrix from its first two rows: the complex
// conjugate of the cofactor, conj(M0i M1j - M0j M1i) with (i, j) = (k+1, k+2)
// mod 3.  m holds rows 0 and 1 row-major (m[3*row + col]).
template <typename T>
__device__ __forceinline__ cplx<T> row2_entry(const cplx<T>* m, int k) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    cplx<T> c = cmul(m[i], m[3 + j]);
    c.x = fma(-m[j].x, m[3 + i].x, c.x);
    c.x = fma(m[j].y, m[3 + i].y, c.x);
    c.y = fma(-m[j].x, m[3 + i].y, c.y);
    c.y = fma(-m[j].y, m[3 + i].x, c.y);
    return mk(c.x, -c.y);
}

__device__ __forceinline__ void c12_load(const float4* __restrict__ src, size_t stride, cplx<float>* m) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 v = src[q * stride];
        m[2 * q] = mk(v.x, v.y);
        m[2 * q + 1] = mk(v.z, v.w);
    }
}
__device__ __forceinline__ void c12_store(float4* __restrict__ dst, size_t stride, const cplx<float>* m) {
#pragma unroll
    for (int q = 0; q < 3; ++q) dst[q * stride] = make_float4(m[2 * q].x, m[2 * q].y, m[2 * q + 1].x, m[2 * q + 1].y);
}

// Re-unitarisation in the compact form (same precision): normalise row 0,
// remove its component from row 1, normalise row 1; row 2 stays implied.
template <typename T>
__device__ __forceinline__ void c12_reunitarise(cplx<T>* m) {
    T n0 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) n0 = fma(m[k].x, m[k].x, fma(m[k].y, m[k].y, n0));
    n0 = rsqrt(n0);
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] = mk(m[k].x * n0, m[k].y * n0);
    T px = T(0), py = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        px = fma(m[k].x, m[3 + k].x, fma(m[k].y, m[3 + k].y, px));
        py = fma(m[k].x, m[3 + k].y, fma(-m[k].y, m[3 + k].x, py));
    }
    T n1 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m[3 + k].x = fma(-px, m[k].x, fma(py, m[k].y, m[3 + k].x));
        m[3 + k].y = fma(-px, m[k].y, fma(-py, m[k].x, m[3 + k].y));
        n1 = fma(m[3 + k].x, m[3 + k].x, fma(m[3 + k].y, m[3 + k].y, n1));
    }
    n1 = rsqrt(n1);
#pragma unroll
    for (int k = 0; k < 3; ++k) m[3 + k] = mk(m[3 + k].x * n1, m[3 + k].y * n1);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async, no register staging)
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (deterministic for a fixed block size); result valid in
// thread 0.  scratch must hold blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) r += scratch[k];
    }
    __syncthreads();
    return r;
}

}  // namespace mcg
