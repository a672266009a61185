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
#include <cstddef>
#include <cmath>
#include <type_traits>
#include <vector>

#include "mcg_common.cuh"
#include "mcg_internal.h"
#include "mcg_sweep.cuh"

namespace mcg {

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
    bool active = s < g.vh;
    int c[4];
    if (active) {
        eo_coords(g, parity, s, c);
        active = c[3] >= fd.t_lo && c[3] < fd.t_hi;  // the sites of a t-slab (whole lattice by default)
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemLinks<T, NT> lk;
    lk.base = reinterpret_cast<cplx<T>*>(smem_raw);

    double rsum = 0.0;
    int fb = 0;
    if (active) {
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

// Haar-random SU(3) matrix of the site with lexicographic index x: Philox4x64-10
// at counters (x, seq, j, 0), j = 0, 1, 2, under key (seed, 0x52414E44) gives
// twelve numbers u in [0, 1); Box-Muller on the pairs (1 - u_2i, u_2i+1)
// gives twelve standard normals, the real and imaginary parts of two complex
// Gaussian rows z0, z1.  Gram-Schmidt makes them rows 0 and 1 of a Haar
// unitary matrix; row 2 = conj(row0 x row1) sets det = 1.
__device__ __noinline__ void haar_su3_site(unsigned long long x, unsigned long long seed, unsigned long long seq,
                                           cplx<double>* m) {
    double u[12];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        unsigned long long c[4] = {x, seq, (unsigned long long)j, 0ull};
        philox4x64_10(c, seed, 0x52414E44ull);
#pragma unroll
        for (int q = 0; q < 4; ++q) u[4 * j + q] = unit_interval(c[q]);
    }
    double n[12];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double r = sqrt(-2.0 * log(1.0 - u[2 * i]));
        double sn, cs;
        sincospi(2.0 * u[2 * i + 1], &sn, &cs);
        n[2 * i] = r * cs;
        n[2 * i + 1] = r * sn;
    }
    cplx<double> r0[3], r1[3];
    double n0 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r0[k] = mk(n[2 * k], n[2 * k + 1]);
        r1[k] = mk(n[6 + 2 * k], n[6 + 2 * k + 1]);
        n0 += r0[k].x * r0[k].x + r0[k].y * r0[k].y;
    }
    const double i0 = 1.0 / sqrt(n0);
    // <r0, z1> = sum conj(r0_k) z1_k
    double pr = 0.0, pi = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r0[k] = mk(r0[k].x * i0, r0[k].y * i0);
        pr += r0[k].x * r1[k].x + r0[k].y * r1[k].y;
        pi += r0[k].x * r1[k].y - r0[k].y * r1[k].x;
    }
    double n1 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r1[k] = mk(r1[k].x - (pr * r0[k].x - pi * r0[k].y), r1[k].y - (pr * r0[k].y + pi * r0[k].x));
        n1 += r1[k].x * r1[k].x + r1[k].y * r1[k].y;
    }
    const double i1 = 1.0 / sqrt(n1);
#pragma unroll
    for (int k = 0; k < 3; ++k) r1[k] = mk(r1[k].x * i1, r1[k].y * i1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m[k] = r0[k];
        m[3 + k] = r1[k];
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        // conj(r0_a r1_b - r0_b r1_a)
        const double re = (r0[a].x * r1[b].x - r0[a].y * r1[b].y) - (r0[b].x * r1[a].x - r0[b].y * r1[a].y);
        const double im = (r0[a].x * r1[b].y + r0[a].y * r1[b].x) - (r0[b].x * r1[a].y + r0[b].y * r1[a].x);
        m[6 + k] = mk(re, -im);
    }
}

// G (FP64, nfields transforms) <- Haar-random SU(3) per site, the same matrices
// in every field (the counter holds the site, not the field)
__global__ void __launch_bounds__(128) k_random_gauge(cplx<double>* __restrict__ G, Geom g, int nfields,
                                                      unsigned long long seed, unsigned long long seq) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    int c[4];
    eo_coords(g, p, s, c);
    const unsigned long long x =
        (unsigned long long)c[0] + (unsigned long long)g.n[0] * (c[1] + (unsigned long long)g.n[1] * (c[2] + (unsigned long long)g.n[2] * c[3]));
    cplx<double> m[9];
    haar_su3_site(x, seed, seq, m);
    cplx<double>* Gf = G + (size_t)f * 18 * g.vh;
#pragma unroll
    for (int e = 0; e < 9; ++e) Gf[gidx(g, p, e, s)] = m[e];
}

// G <- W G per site (FP64; W one field, applied to each of the nfields)
__global__ void __launch_bounds__(128) k_gauge_left_mul(cplx<double>* __restrict__ G, const cplx<double>* __restrict__ W,
                                                        Geom g, int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    cplx<double>* Gf = G + (size_t)f * 18 * g.vh;
    cplx<double> a[9], b[9], o[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        a[e] = W[gidx(g, p, e, s)];
        b[e] = Gf[gidx(g, p, e, s)];
    }
    m3_mul(a, b, o);
#pragma unroll
    for (int e = 0; e < 9; ++e) Gf[gidx(g, p, e, s)] = o[e];
}

int launch_random_gauge(void* G, const Geom& g, int nfields, unsigned long long seed, unsigned long long seq,
                        cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    if (n <= 0) return 0;
    k_random_gauge<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((cplx<double>*)G, g, nfields, seed, seq);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_gauge_left_mul(void* G, const void* W, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    if (n <= 0) return 0;
    k_gauge_left_mul<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((cplx<double>*)G, (const cplx<double>*)W, g,
                                                                  nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

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
    // each thread adds its strided partials k, k + blockDim, ... in that
    // order; eight are loaded before they are added (zeros past the end come
    // after the last partial, so the sum is unchanged), which takes the
    // dependent load latency off this kernel: it sits on the critical path of
    // every sweep (measured: a lone-field fix 4 % faster, same bits)
    for (size_t k = threadIdx.x; k < n; k += 8 * (size_t)blockDim.x) {
        double x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const size_t kk = k + (size_t)j * blockDim.x;
            x[j] = kk < n ? part[kk] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) v += x[j];
    }
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

// sum of n partials in a fixed order (one block)
__global__ void __launch_bounds__(256) k_sum_slab_partials(const double* __restrict__ partial, int n,
                                                           double* __restrict__ out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partial[k];
    __shared__ double red[8];
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) *out = tot;
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
        int rc = 0;
        if ((rc = prepare_halfsweep_c12(nt))) return rc;
    }
    return 0;
}

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
        launch_halfsweep_c12(nt, acc, bt, parity, nblocks, st);
    }
}

template <typename T>
static int enqueue_sweep(const SweepBatch& bt, int nt, int spb, cudaStream_t st) {
    if constexpr (std::is_same<T, DoubleFloat>::value) {
        // no re-unitarisation inside the phase: the double-float links drift
        // from unitarity by ~1e-14 per sweep; the output is the FP64 field
        // transformed by the re-unitarised W of the phase
        launch_halfsweep_df(false, bt, 0, bt.total_blocks, st);
        launch_halfsweep_df(true, bt, 1, bt.total_blocks, st);
        k_finalize<<<bt.nf, 256, 0, st>>>(bt, 0);
    } else {
        launch_halfsweep<T>(nt, false, bt, 0, bt.total_blocks, st);
        launch_halfsweep<T>(nt, true, bt, 1, bt.total_blocks, st);
        k_finalize<<<bt.nf, 256, 0, st>>>(bt, 0);
        // FP32 sweeps re-unitarise inside the half-sweep kernel
        if constexpr (sizeof(T) == 8)
            if (bt.reunit_every > 0) k_reunit_pending<T><<<bt.total_blocks, spb, 0, st>>>(bt);
    }
    return 0;
}

// largest batch captured as per-field chains
constexpr int kMaxChains = 16;

template <typename T>
int run_fix_phase(const std::vector<FieldDesc>& fields_in, FieldState* d_state, FieldState* h_state, double* d_hist,
                  int hist_len, double tol, int window, double omega, int reunit_every, int abs_cap,
                  int check_every, bool fresh, cudaStream_t stream, bool solve32, const PhaseRestart* restart) {
    constexpr bool DF = std::is_same<T, DoubleFloat>::value;
    const int prec = (DF || sizeof(T) == 8) ? MCG_F64 : MCG_F32;
    const int NT = DF ? df_threads() : sweep_block(prec);
    const int SPB = DF ? NT : sweep_sites_per_block(prec);
    const int nf = (int)fields_in.size();
    std::vector<FieldDesc> fields = fields_in;
    int total = 0;
    for (auto& fd : fields) {
        fd.nblk = (fd.geo.vh + SPB - 1) / SPB;
        fd.blk0 = total;
        fd.omega = omega;
        total += fd.nblk;
    }
    const bool restarts = restart && (restart->after > 0 || restart->creep > 0) && std::is_same<T, float>::value;
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

    if constexpr (DF) {
        if ((rc = prepare_halfsweep_df())) return rc;
        launch_functional_df(bt, total, stream);
    } else {
        if ((rc = prepare_halfsweep<T>(NT))) return rc;
        k_functional<T><<<total, SPB, 0, stream>>>(bt);
    }
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
    // A batch of a few fields runs as independent per-field chains of
    // half-sweeps inside the graph (one branch stream each, forked from and
    // joined to the capture stream): no field waits for another at the
    // half-sweep boundaries, the fields drift apart in phase, and one field's
    // load phase overlaps another's arithmetic (measured: the step 4.6 %
    // faster than one launch per half-sweep covering every field).  Each chain
    // sees its field as a batch of one (block offset 0, its own state, partials
    // and R history), so the per-field arithmetic is unchanged.  A large batch
    // fills the GPU with one launch per half-sweep and keeps the graph small.
    const bool chained = nf > 1 && nf <= kMaxChains;
    std::vector<SweepBatch> chains;
    std::vector<cudaStream_t> bs(nf);
    std::vector<cudaEvent_t> be(nf);
    cudaEvent_t fork = nullptr;
    // each field as a batch of one (the chains, and the R of a restarted field)
    FieldDesc* d_single = nullptr;
    if (chained || restarts) {
        d_single = (FieldDesc*)scratch_device("fix.desc1", sizeof(FieldDesc) * nf, &rc);
        if (rc) return rc;
        FieldDesc* h_single = (FieldDesc*)scratch_host("fix.desc1", sizeof(FieldDesc) * nf, &rc);
        if (rc) return rc;
        for (int f = 0; f < nf; ++f) {
            h_single[f] = fields[f];
            h_single[f].blk0 = 0;
        }
        MCG_CK(cudaMemcpyAsync(d_single, h_single, sizeof(FieldDesc) * nf, cudaMemcpyHostToDevice, stream));
        MCG_CK(cudaStreamSynchronize(stream));  // h_single is reused by the next call
        for (int f = 0; f < nf; ++f) {
            SweepBatch b = bt;
            b.desc = d_single + f;
            b.nf = 1;
            b.total_blocks = fields[f].nblk;
            b.state = d_state + f;
            b.partial = d_partial + (size_t)fields[f].blk0 * bt.ppb;
            b.R_hist = d_hist ? d_hist + (size_t)f * hist_len : nullptr;
            chains.push_back(b);
        }
        if (chained && branch_streams(nf, bs.data(), be.data(), &fork, &rc)) return rc;
    }
    MCG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    // no early return while the capture is open: the first error ends it
    cudaError_t qe = cudaSuccess;
    if (chained) {
        qe = cudaEventRecord(fork, cs);
        for (int f = 0; f < nf && qe == cudaSuccess; ++f) {
            qe = cudaStreamWaitEvent(bs[f], fork, 0);
            if (qe != cudaSuccess) break;
            for (int i = 0; i < chunk; ++i) enqueue_sweep<T>(chains[f], NT, SPB, bs[f]);
            qe = cudaEventRecord(be[f], bs[f]);
            if (qe == cudaSuccess) qe = cudaStreamWaitEvent(cs, be[f], 0);
        }
    } else {
        for (int i = 0; i < chunk; ++i) enqueue_sweep<T>(bt, NT, SPB, cs);
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (qe != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(qe != cudaSuccess ? qe : ce, "sweep graph capture");
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ce, "cudaGraphInstantiate");
    }
    const int nodes_per_chunk = (chained ? nf : 1) * chunk * ((!DF && sizeof(T) == 8 && reunit_every > 0) ? 4 : 3);
    const int max_chunks = (phase_len + chunk - 1) / chunk + 1;
    int status = 0;
    // The next chunk is launched before the host reads the state after the
    // current one, so the GPU does not wait for the host between chunks: a
    // field that is done makes every later kernel of its chain exit at entry,
    // so a chunk launched after the last field finished sweeps nothing and the
    // results are those of launching chunk by chunk.  The state after each
    // chunk is copied to one of two pinned buffers.  Phase timing
    // (instrumentation): GPU time of the chunk graphs and the site-updates
    // they performed.
    FieldState* h_ring = (FieldState*)scratch_host("fix.state2", sizeof(FieldState) * 2 * nf, &rc);
    cudaEvent_t t0[2] = {nullptr, nullptr}, t1[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    bool evs = rc == 0;
    for (int i = 0; i < 2 && evs; ++i)
        evs = cudaEventCreate(&t0[i]) == cudaSuccess && cudaEventCreate(&t1[i]) == cudaSuccess &&
              cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming) == cudaSuccess;
    auto launch = [&](int c) -> cudaError_t {
        const int b = c & 1;
        cudaError_t e = cudaEventRecord(t0[b], stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream);
        if (e == cudaSuccess) e = cudaEventRecord(t1[b], stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_ring + (size_t)b * nf, d_state, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost,
                                stream);
        if (e == cudaSuccess) e = cudaEventRecord(copied[b], stream);
        if (e == cudaSuccess) note_launches(nodes_per_chunk);
        return e;
    };
    std::vector<int> sw0(nf);
    for (int f = 0; f < nf; ++f) sw0[f] = h_state[f].sweep;
    // restarts: each field's restarts, the first chunk whose state read
    // follows its last reset, and a pinned slot per field for the
    // over-relaxation written to its descriptors.  A field's (re)start is its
    // state's phase_start.
    std::vector<int> nrestart(nf, 0), valid_from(nf, 0);
    // the creep test: per field, the per-chunk dV_U since its (re)start (a
    // ring of the last m chunks) and the R and sweep count of its last read
    const int creep_m = (restarts && restart->creep > 0) ? std::max(4, restart->creep / chunk) : 0;
    std::vector<double> creep_dv((size_t)nf * std::max(creep_m, 1), 0.0), last_R(nf, 0.0);
    std::vector<int> creep_n(nf, 0), last_sweep(nf, -1);
    double* h_omega = nullptr;
    if (restarts) {
        h_omega = (double*)scratch_host("fix.restart.omega", sizeof(double) * nf, &rc);
        if (rc) status = rc;
    }
    // enqueue the reset of field f after the chunk in flight (stream order)
    auto restart_field = [&](int f, double om) -> int {
        int r = restart->reset(f, nrestart[f] + 1, stream);
        if (r) return r;
        h_omega[f] = om;
        const size_t off = offsetof(FieldDesc, omega);
        cudaError_t e = cudaMemcpyAsync((char*)(d_desc + f) + off, h_omega + f, sizeof(double),
                                        cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)(d_single + f) + off, h_omega + f, sizeof(double), cudaMemcpyHostToDevice,
                                stream);
        if (e != cudaSuccess) return cuda_fail(e, "restart descriptors");
        // R of the reset field and a new phase start for it (its sweep count
        // goes on)
        if constexpr (std::is_same<T, float>::value) {
            k_functional<T><<<fields[f].nblk, SPB, 0, stream>>>(chains[f]);
            k_finalize<<<1, 256, 0, stream>>>(chains[f], 2);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "restart");
            note_launches(2);
        }
        return 0;
    };
    int in_flight = -1;  // a chunk launched after the last one read
    if (!evs) {
        status = rc ? rc : fail(MCG_CUDA_ERROR, "sweep chunk events");
    } else if ((ce = launch(0)) != cudaSuccess) {
        status = cuda_fail(ce, "cudaGraphLaunch");
    }
    for (int c = 0; status == 0 && c < max_chunks; ++c) {
        const int b = c & 1;
        in_flight = -1;
        if (c + 1 < max_chunks) {
            if ((ce = launch(c + 1)) != cudaSuccess) {
                status = cuda_fail(ce, "cudaGraphLaunch");
                break;
            }
            in_flight = c + 1;
        }
        if ((ce = cudaEventSynchronize(copied[b])) != cudaSuccess) {
            status = cuda_fail(ce, "sweep chunk");
            break;
        }
        const FieldState* hs = h_ring + (size_t)b * nf;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0[b], t1[b]);
        long long su = 0;
        for (int f = 0; f < nf; ++f) {
            su += (long long)(hs[f].sweep - sw0[f]) * 2LL * fields[f].geo.vh;
            sw0[f] = hs[f].sweep;
        }
        note_phase(prec, ms, su);
        bool all = true;
        for (int f = 0; f < nf; ++f) {
            if (c < valid_from[f]) {
                all = false;  // a reset is pending behind the chunk read here
                continue;
            }
            bool creeps = false;
            if (creep_m > 0 && hs[f].done == 0) {
                if (last_sweep[f] >= 0 && hs[f].sweep > last_sweep[f]) {
                    double* ring = creep_dv.data() + (size_t)f * creep_m;
                    ring[creep_n[f] % creep_m] =
                        (hs[f].R_last - last_R[f]) * fields[f].norm / (hs[f].sweep - last_sweep[f]);
                    ++creep_n[f];
                    if (creep_n[f] >= creep_m) {
                        std::vector<double> w(creep_m);
                        for (int i = 0; i < creep_m; ++i) w[i] = ring[(creep_n[f] + i) % creep_m];
                        creeps = creeping(w.data(), creep_m, restart->creep_lo, restart->creep_hi);
                    }
                }
                last_R[f] = hs[f].R_last;
                last_sweep[f] = hs[f].sweep;
            }
            if (restarts && hs[f].done == 0 &&
                ((restart->after > 0 && hs[f].sweep - hs[f].phase_start >= restart->after) || creeps)) {
                const double om = restart_omega(omega, restart->domega, nrestart[f] + 1);
                if (om > 0.0 && om < 2.0 && in_flight == c + 1) {
                    if ((rc = restart_field(f, om))) {
                        status = rc;
                        break;
                    }
                    ++nrestart[f];
                    valid_from[f] = c + 2;
                    creep_n[f] = 0;
                    last_sweep[f] = -1;
                    all = false;
                    continue;
                }
            }
            all = all && hs[f].done != 0;
        }
        if (status) break;
        if (all) break;
    }
    if (restarts && restart->count)
        for (int f = 0; f < nf; ++f) restart->count[f] = nrestart[f];
    // the chunk still in flight (if any) sweeps nothing once every field is
    // done; its GPU time is counted with the phase
    ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess && status == 0) status = cuda_fail(ce, "sweep chunk");
    if (status == 0 && in_flight >= 0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t0[in_flight & 1], t1[in_flight & 1]) == cudaSuccess) note_phase(prec, ms, 0);
    }
    // the caller's copy of the state after the phase
    if (status == 0) {
        ce = cudaMemcpyAsync(h_state, d_state, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) status = cuda_fail(ce, "sweep state");
    }
    for (int i = 0; i < 2; ++i) {
        if (t0[i]) cudaEventDestroy(t0[i]);
        if (t1[i]) cudaEventDestroy(t1[i]);
        if (copied[i]) cudaEventDestroy(copied[i]);
    }
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

int run_halfsweep_slab(void* U, void* G, const Geom& g, int parity, int t_lo, int t_hi, bool want_R, double* R_host,
                       cudaStream_t stream) {
    const int NT = sweep_block(MCG_F64);
    int rc = 0;
    FieldDesc fd;
    fd.U = U;
    fd.G = G;
    fd.geo = g;
    fd.blk0 = 0;
    fd.nblk = (g.vh + NT - 1) / NT;
    fd.norm = 1.0 / (9.0 * 8.0 * g.vh);
    fd.t_lo = t_lo;
    fd.t_hi = t_hi;
    FieldDesc* d_desc = (FieldDesc*)scratch_device("slab.desc", sizeof(FieldDesc), &rc);
    if (rc) return rc;
    FieldState* d_state = (FieldState*)scratch_device("slab.state", sizeof(FieldState), &rc);
    if (rc) return rc;
    double* d_partial = (double*)scratch_device("slab.partial", sizeof(double) * fd.nblk * (NT / 32), &rc);
    if (rc) return rc;
    double* d_R = (double*)scratch_device("slab.R", sizeof(double), &rc);
    if (rc) return rc;
    FieldDesc* h_desc = (FieldDesc*)scratch_host("slab.desc", sizeof(FieldDesc), &rc);
    if (rc) return rc;
    MCG_CK(cudaStreamSynchronize(stream));  // the previous call may still read the staging buffer
    *h_desc = fd;
    MCG_CK(cudaMemcpyAsync(d_desc, h_desc, sizeof fd, cudaMemcpyHostToDevice, stream));
    MCG_CK(cudaMemsetAsync(d_state, 0, sizeof(FieldState), stream));
    SweepBatch bt;
    bt.desc = d_desc;
    bt.nf = 1;
    bt.total_blocks = fd.nblk;
    bt.state = d_state;
    bt.partial = d_partial;
    bt.ppb = NT / 32;
    bt.R_hist = nullptr;
    bt.hist_len = 0;
    bt.tol = 0;
    bt.window = 1;
    bt.reunit_every = 0;
    bt.omega = 1.0;
    bt.solve32 = 0;
    if ((rc = prepare_halfsweep<double>(NT))) return rc;
    launch_halfsweep<double>(NT, want_R, bt, parity, fd.nblk, stream);
    note_launches(1);
    MCG_CK(cudaGetLastError());
    if (want_R) {
        k_sum_slab_partials<<<1, 256, 0, stream>>>(d_partial, fd.nblk * (NT / 32), d_R);
        note_launches(1);
        MCG_CK(cudaGetLastError());
        MCG_CK(cudaMemcpyAsync(R_host, d_R, sizeof(double), cudaMemcpyDeviceToHost, stream));
        MCG_CK(cudaStreamSynchronize(stream));
    }
    return 0;
}

// One local problem per thread (the subgroup maximisation on its own): the
// solve of the FP32 sweeps (A, b rounded to FP32; certified Newton, else the
// FP32 Jacobi + secular path) or that of the exact FP64 sweep.
__global__ void __launch_bounds__(128) k_local_solve(const double* __restrict__ A16, const double* __restrict__ b4,
                                                     double* __restrict__ a4, int* __restrict__ fb, int n, int prec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double A[4][4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        b[i] = b4[4 * (size_t)k + i];
#pragma unroll
        for (int j = i; j < 4; ++j) A[i][j] = A[j][i] = A16[16 * (size_t)k + 4 * i + j];
    }
    double a[4];
    int f = 0;
    if (prec == MCG_F32) {
        float Af[4][4], bf[4], af[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            bf[i] = (float)b[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) Af[i][j] = (float)A[i][j];
        }
        if (!kkt_newton_f32(Af, bf, af)) {
            const float4 r = solve_f32_fallback(Af[0][0], Af[0][1], Af[0][2], Af[0][3], Af[1][1], Af[1][2], Af[1][3],
                                                Af[2][2], Af[2][3], Af[3][3], bf[0], bf[1], bf[2], bf[3]);
            af[0] = r.x;
            af[1] = r.y;
            af[2] = r.z;
            af[3] = r.w;
            f = 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = (double)af[i];
    } else {
        f = Solver<double>::solve(A, b, a);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) a4[4 * (size_t)k + i] = a[i];
    if (fb) fb[k] = f;
}

int launch_local_solve(const double* A16, const double* b4, double* a4, int* fb, int n, int prec, cudaStream_t st) {
    if (n <= 0) return 0;
    k_local_solve<<<(n + 127) / 128, 128, 0, st>>>(A16, b4, a4, fb, n, prec);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

template int time_halfsweep<float>(void*, void*, const Geom&, int, int, int, float*, cudaStream_t);
template int time_halfsweep<double>(void*, void*, const Geom&, int, int, int, float*, cudaStream_t);

template int run_fix_phase<float>(const std::vector<FieldDesc>&, FieldState*, FieldState*, double*, int, double,
                                  int, double, int, int, int, bool, cudaStream_t, bool, const PhaseRestart*);
template int run_fix_phase<DoubleFloat>(const std::vector<FieldDesc>&, FieldState*, FieldState*, double*, int,
                                        double, int, double, int, int, int, bool, cudaStream_t, bool,
                                        const PhaseRestart*);
template int run_fix_phase<double>(const std::vector<FieldDesc>&, FieldState*, FieldState*, double*, int, double,
                                   int, double, int, int, int, bool, cudaStream_t, bool, const PhaseRestart*);

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_sweep)

}  // namespace mcg
