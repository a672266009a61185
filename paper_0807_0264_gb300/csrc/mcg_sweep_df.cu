// FP64-class MCG sweeps in double-float arithmetic (the final sweeps of the
// mixed-precision schedule with mcg_params.fp64_df = 1).
//
// GB300 executes FP64 at about 1/60 of its FP32 rate (conversions between the
// two included), and the FP64 half-sweep spends ~75 % of its time in the FP64
// pipe.  Here a link entry is held as a pair of FP32 numbers hi + lo with
// |lo| <= ulp(hi)/2 (a 48-bit significand), in the compact storage (rows 0 and
// 1 of each matrix, row 2 implied by unitarity): hi chunks in the c12 layout
// of the FP32 sweeps, lo chunks in a second array of the same layout.  The
// SU(2) moves are applied with error-free transformations on the FP32 pipe:
// Knuth's two-sum and the FMA two-product (Dekker 1971), so each entry keeps
// ~1e-14 relative accuracy per operation.  The local 4x4 problem is built and
// solved in FP32 from the hi parts, as in the fp64_solve32 FP64 sweeps; its
// solution is normalised in FP64 (so G is unitary to FP64 precision) and split
// into double-float.  The functional R is accumulated in double-float per site
// and in FP64 across sites, so the stop rule dV_U < tol is an FP64 test.  The
// field's own FP64 links are not touched during the phase: the transform W of
// the phase is accumulated in double-float and applied to them in FP64 at the
// end (re-unitarised), which keeps the output exactly on its gauge orbit.
#include <cuda_runtime.h>

#include "mcg_common.cuh"
#include "mcg_internal.h"
#include "mcg_sweep.cuh"

namespace mcg {

// ---------------------------------------------------------------------------
// double-float arithmetic: a real is float2 (x = hi, y = lo)
// ---------------------------------------------------------------------------
// (sh, sl) = a * b, an unnormalised pair: exact product of the hi parts
// (FMA two-product) plus the cross terms (the lo * lo term is below 2^-48).
__device__ __forceinline__ void dd_first(float& sh, float& sl, float2 a, float2 b) {
    sh = a.x * b.x;
    sl = fmaf(a.x, b.x, -sh);
    sl = fmaf(a.x, b.y, fmaf(a.y, b.x, sl));
}
// (sh, sl) += a * b: the product as above, its hi part added to sh by
// two-sum, every rounding error collected in sl.
__device__ __forceinline__ void dd_mac(float& sh, float& sl, float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float t = sh + p;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sh = t;
    sl += err + e;
}
// (sh, sl) += a: two-sum on the hi parts.
__device__ __forceinline__ void dd_add(float& sh, float& sl, float2 a) {
    const float t = sh + a.x;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (a.x - z);
    sh = t;
    sl += err + a.y;
}
// renormalise (fast two-sum, |sh| >= |sl|)
__device__ __forceinline__ float2 dd_norm(float sh, float sl) {
    const float h = sh + sl;
    return make_float2(h, sl - (h - sh));
}
__device__ __forceinline__ float2 dd_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double dd_to_double(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 dd_from_double(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

struct DC {  // double-float complex
    float2 re, im;
};

// entry (2, k) of an SU(3) matrix from rows 0 and 1: conj(M0i M1j - M0j M1i),
// (i, j) = (k+1, k+2) mod 3
__device__ __forceinline__ DC dc_row2(const DC* m, int k) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    const DC a = m[i], b = m[3 + j], c = m[j], d = m[3 + i];
    float rh, rl, ih, il;
    dd_first(rh, rl, a.re, b.re);
    dd_mac(rh, rl, dd_neg(a.im), b.im);
    dd_mac(rh, rl, dd_neg(c.re), d.re);
    dd_mac(rh, rl, c.im, d.im);
    dd_first(ih, il, a.re, b.im);
    dd_mac(ih, il, a.im, b.re);
    dd_mac(ih, il, dd_neg(c.re), d.im);
    dd_mac(ih, il, dd_neg(c.im), d.re);
    return DC{dd_norm(rh, rl), dd_neg(dd_norm(ih, il))};
}

// ---------------------------------------------------------------------------
// The moves on (re, im) lane pairs: one packed FP32 instruction (__ffma2_rn,
// __fmul2_rn, __fadd2_rn) performs the operation of the real and of the
// imaginary chain, each lane exactly as the scalar dd_first / dd_mac /
// dd_norm above (a - b as a + (-b), exact), with half the instructions of two
// scalar chains (measured: the double-float sweep 9 % faster, same bits).  A packed double-float
// complex holds hi = (re.hi, im.hi) and lo = (re.lo, im.lo), which is how the
// hi and lo chunks store an entry.
// ---------------------------------------------------------------------------
struct DCp {
    float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ DCp to_p(const DC& a) {
    return DCp{make_float2(a.re.x, a.im.x), make_float2(a.re.y, a.im.y)};
}
__device__ __forceinline__ DC from_p(const DCp& a) {
    return DC{make_float2(a.hi.x, a.lo.x), make_float2(a.hi.y, a.lo.y)};
}
// lane-wise dd_first (a: ah + al, b: bh + bl)
__device__ __forceinline__ void pdd_first(float2& sh, float2& sl, float2 ah, float2 al, float2 bh, float2 bl) {
    sh = __fmul2_rn(ah, bh);
    sl = __ffma2_rn(ah, bh, neg2(sh));
    sl = __ffma2_rn(ah, bl, __ffma2_rn(al, bh, sl));
}
// lane-wise dd_mac
__device__ __forceinline__ void pdd_mac(float2& sh, float2& sl, float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(ah, bh);
    float2 e = __ffma2_rn(ah, bh, neg2(p));
    e = __ffma2_rn(ah, bl, __ffma2_rn(al, bh, e));
    const float2 t = __fadd2_rn(sh, p);
    const float2 z = sub2(t, sh);
    const float2 err = __fadd2_rn(sub2(sh, sub2(t, z)), sub2(p, z));
    sh = t;
    sl = __fadd2_rn(sl, __fadd2_rn(err, e));
}
__device__ __forceinline__ DCp pdd_norm(float2 sh, float2 sl) {
    const float2 h = __fadd2_rn(sh, sl);
    return DCp{h, sub2(sl, sub2(h, sh))};
}
// coefficient pairs of one SU(2) element entry g: (re, re) and (-im, im) for
// g x, (im, im) for x conj(g)
struct PGc {
    float2 re_h, re_l, nim_h, nim_l, im_h, im_l;
};
__device__ __forceinline__ PGc pg_of(const DC& g) {
    return PGc{make_float2(g.re.x, g.re.x), make_float2(g.re.y, g.re.y), make_float2(-g.im.x, g.im.x),
               make_float2(-g.im.y, g.im.y), make_float2(g.im.x, g.im.x), make_float2(g.im.y, g.im.y)};
}
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }
// g1 u + g2 v: real lane g1.re u.re - g1.im u.im + g2.re v.re - g2.im v.im,
// imaginary lane g1.re u.im + g1.im u.re + g2.re v.im + g2.im v.re
__device__ __forceinline__ DCp pdc_lin(const PGc& g1, const DCp& u, const PGc& g2, const DCp& v) {
    float2 sh, sl;
    pdd_first(sh, sl, g1.re_h, g1.re_l, u.hi, u.lo);
    pdd_mac(sh, sl, g1.nim_h, g1.nim_l, swap2(u.hi), swap2(u.lo));
    pdd_mac(sh, sl, g2.re_h, g2.re_l, v.hi, v.lo);
    pdd_mac(sh, sl, g2.nim_h, g2.nim_l, swap2(v.hi), swap2(v.lo));
    return pdd_norm(sh, sl);
}
// (im, -re) of a pair
__device__ __forceinline__ float2 swapneg2(float2 a) { return make_float2(a.y, -a.x); }
// u conj(g1) + v conj(g2): real lane u.re g1.re + u.im g1.im + v.re g2.re +
// v.im g2.im, imaginary lane u.im g1.re - u.re g1.im + v.im g2.re - v.re g2.im
__device__ __forceinline__ DCp pdc_lin_conj(const DCp& u, const PGc& g1, const DCp& v, const PGc& g2) {
    float2 sh, sl;
    pdd_first(sh, sl, u.hi, u.lo, g1.re_h, g1.re_l);
    pdd_mac(sh, sl, swapneg2(u.hi), swapneg2(u.lo), g1.im_h, g1.im_l);
    pdd_mac(sh, sl, v.hi, v.lo, g2.re_h, g2.re_l);
    pdd_mac(sh, sl, swapneg2(v.hi), swapneg2(v.lo), g2.im_h, g2.im_l);
    return pdd_norm(sh, sl);
}

// ---------------------------------------------------------------------------
// the site's 9 matrices in shared memory: chunk (part, mat, q) of thread t at
// S[((part * 9 + mat) * 3 + q) * NT + t], part 0 = hi, 1 = lo; mat 0..3 the
// forward links U_mu(x), 4..7 the backward links U_mu(x - mu), 8 the transform
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void dc_load(const float4* S, int mat, DC (&m)[6]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 h = S[((0 * 9 + mat) * 3 + q) * NT + threadIdx.x];
        const float4 l = S[((1 * 9 + mat) * 3 + q) * NT + threadIdx.x];
        m[2 * q] = DC{make_float2(h.x, l.x), make_float2(h.y, l.y)};
        m[2 * q + 1] = DC{make_float2(h.z, l.z), make_float2(h.w, l.w)};
    }
}
template <int NT>
__device__ __forceinline__ void dc_store(float4* S, int mat, const DC (&m)[6]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        S[((0 * 9 + mat) * 3 + q) * NT + threadIdx.x] =
            make_float4(m[2 * q].re.x, m[2 * q].im.x, m[2 * q + 1].re.x, m[2 * q + 1].im.x);
        S[((1 * 9 + mat) * 3 + q) * NT + threadIdx.x] =
            make_float4(m[2 * q].re.y, m[2 * q].im.y, m[2 * q + 1].re.y, m[2 * q + 1].im.y);
    }
}
template <int NT>
__device__ __forceinline__ void dcp_load(const float4* S, int mat, DCp (&m)[6]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 h = S[((0 * 9 + mat) * 3 + q) * NT + threadIdx.x];
        const float4 l = S[((1 * 9 + mat) * 3 + q) * NT + threadIdx.x];
        m[2 * q] = DCp{make_float2(h.x, h.y), make_float2(l.x, l.y)};
        m[2 * q + 1] = DCp{make_float2(h.z, h.w), make_float2(l.z, l.w)};
    }
}
template <int NT>
__device__ __forceinline__ void dcp_store(float4* S, int mat, const DCp (&m)[6]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        S[((0 * 9 + mat) * 3 + q) * NT + threadIdx.x] =
            make_float4(m[2 * q].hi.x, m[2 * q].hi.y, m[2 * q + 1].hi.x, m[2 * q + 1].hi.y);
        S[((1 * 9 + mat) * 3 + q) * NT + threadIdx.x] =
            make_float4(m[2 * q].lo.x, m[2 * q].lo.y, m[2 * q + 1].lo.x, m[2 * q + 1].lo.y);
    }
}
// M <- G M on rows (P, Q) of a compact matrix; for Q = 2 only row P is stored
// (row 2 rebuilt by the scalar cofactor, which reads the same registers)
template <int P, int Q>
__device__ __forceinline__ void dcp_left(DCp (&m)[6], const PGc (&g)[4]) {
    if constexpr (Q < 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const DCp xp = m[3 * P + k], xq = m[3 * Q + k];
            m[3 * P + k] = pdc_lin(g[0], xp, g[1], xq);
            m[3 * Q + k] = pdc_lin(g[2], xp, g[3], xq);
        }
    } else {
        DC ms[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) ms[k] = from_p(m[k]);
        DCp r2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) r2[k] = to_p(dc_row2(ms, k));
#pragma unroll
        for (int k = 0; k < 3; ++k) m[3 * P + k] = pdc_lin(g[0], m[3 * P + k], g[1], r2[k]);
    }
}

// hi parts only, as FP32 complex (the local problem is built from them)
template <int NT>
__device__ __forceinline__ void hi_load(const float4* S, int mat, cplx<float> (&m)[6]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 h = S[(mat * 3 + q) * NT + threadIdx.x];
        m[2 * q] = mk(h.x, h.y);
        m[2 * q + 1] = mk(h.z, h.w);
    }
}

template <int I, int J>
__device__ __forceinline__ cplx<float> hi_entry(const cplx<float>* m) {
    if constexpr (I < 2)
        return m[3 * I + J];
    else
        return row2_entry(m, J);
}

// One SU(2)-subgroup step on the site's matrices in shared memory: (A, b)
// from the hi parts (FP32), the FP32 local solve, the solution normalised in
// FP64 and split, the move applied in double-float.  Returns 1 if the solve
// left the Newton path.
template <int P, int Q, int R, int NT>
__device__ __forceinline__ int df_subgroup_step(float4* S) {
    float2 Ap[10], bp[4];
#pragma unroll
    for (int i = 0; i < 10; ++i) Ap[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) bp[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        cplx<float> M[6];
        hi_load<NT>(S, l, M);
        const cplx<float> m11 = hi_entry<P, P>(M), m12 = hi_entry<P, Q>(M);
        const cplx<float> m21 = hi_entry<Q, P>(M), m22 = hi_entry<Q, Q>(M);
        const cplx<float> cc = hi_entry<R, R>(M);
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
    float a[4];
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
    // G unitary to FP64 precision: the FP32 solution normalised in FP64
    double ad[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ad[k] = (double)a[k];
    const double inv = rsqrt(ad[0] * ad[0] + ad[1] * ad[1] + ad[2] * ad[2] + ad[3] * ad[3]);
    float2 af[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) af[k] = dd_from_double(ad[k] * inv);
    // G = (a0 + i a3, a2 + i a1; -a2 + i a1, a0 - i a3): g11, g12, g21, g22
    const DC g[4] = {DC{af[0], af[3]}, DC{af[2], af[1]}, DC{dd_neg(af[2]), af[1]}, DC{af[0], dd_neg(af[3])}};
    const PGc gp[4] = {pg_of(g[0]), pg_of(g[1]), pg_of(g[2]), pg_of(g[3])};
    // forward links and the transform: rows P, Q of G M
#pragma unroll 1
    for (int l = 0; l < 5; ++l) {
        const int mat = l < 4 ? l : 8;
        DCp m[6];
        dcp_load<NT>(S, mat, m);
        dcp_left<P, Q>(m, gp);
        dcp_store<NT>(S, mat, m);
    }
    // backward links: columns P, Q of M G^dag, rows 0 and 1
#pragma unroll 1
    for (int l = 4; l < 8; ++l) {
        DCp m[6];
        dcp_load<NT>(S, l, m);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const DCp xp = m[3 * i + P], xq = m[3 * i + Q];
            m[3 * i + P] = pdc_lin_conj(xp, gp[0], xq, gp[1]);
            m[3 * i + Q] = pdc_lin_conj(xp, gp[2], xq, gp[3]);
        }
        dcp_store<NT>(S, l, m);
    }
    return fb;
}

// |tr M|^2 in double-float, added to (sh, sl)
template <int NT>
__device__ __forceinline__ void df_trace2(const float4* S, int mat, float& sh, float& sl) {
    DC m[6];
    dc_load<NT>(S, mat, m);
    const DC r22 = dc_row2(m, 2);
    float th, tl, uh, ul;
    th = m[0].re.x;
    tl = m[0].re.y;
    dd_add(th, tl, m[4].re);
    dd_add(th, tl, r22.re);
    uh = m[0].im.x;
    ul = m[0].im.y;
    dd_add(uh, ul, m[4].im);
    dd_add(uh, ul, r22.im);
    const float2 tr = dd_norm(th, tl), ti = dd_norm(uh, ul);
    dd_mac(sh, sl, tr, tr);
    dd_mac(sh, sl, ti, ti);
}

constexpr int kDFThreads = 64;

// One thread per site; the 9 matrices of the site (hi and lo, 54 chunks,
// 864 bytes) staged in shared memory by cp.async: 55 KB per block of 64.
template <bool ACC, int NT>
__global__ void __launch_bounds__(NT, 4) k_halfsweep_df(SweepBatch bt, int parity) {
    extern __shared__ float4 df_smem[];
    float4* S = df_smem;
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    if (bt.state[f].done) return;  // block-uniform
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    float4* __restrict__ Uh = reinterpret_cast<float4*>(fd.U);
    float4* __restrict__ Ul = reinterpret_cast<float4*>(fd.Ulo);
    float4* __restrict__ Wh = reinterpret_cast<float4*>(fd.G);
    float4* __restrict__ Wl = reinterpret_cast<float4*>(fd.Glo);
    const int s = (blockIdx.x - fd.blk0) * NT + threadIdx.x;
    double rsum = 0.0;
    int fb = 0;
    if (s < g.vh) {
        int c[4];
        eo_coords(g, parity, s, c);
        int sb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) sb[mu] = eo_neighbor(g, c, mu, -1);
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const float4* Ub = part ? Ul : Uh;
            const float4* Wb = part ? Wl : Wh;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    cp_async<16>(&S[((part * 9 + mu) * 3 + q) * NT + threadIdx.x], Ub + c12_lidx(g, mu, parity, q, s));
                    cp_async<16>(&S[((part * 9 + 4 + mu) * 3 + q) * NT + threadIdx.x],
                                 Ub + c12_lidx(g, mu, parity ^ 1, q, sb[mu]));
                }
#pragma unroll
            for (int q = 0; q < 3; ++q)
                cp_async<16>(&S[((part * 9 + 8) * 3 + q) * NT + threadIdx.x], Wb + c12_gidx(g, parity, q, s));
        }
        cp_async_wait_all();

        fb += df_subgroup_step<0, 1, 2, NT>(S);
        fb += df_subgroup_step<0, 2, 1, NT>(S);
        fb += df_subgroup_step<1, 2, 0, NT>(S);

        if (ACC) {
            float sh = 0.f, sl = 0.f;
#pragma unroll 1
            for (int l = 0; l < 8; ++l) df_trace2<NT>(S, l, sh, sl);
            rsum = (double)sh + (double)sl;
        }
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            float4* Ub = part ? Ul : Uh;
            float4* Wb = part ? Wl : Wh;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    Ub[c12_lidx(g, mu, parity, q, s)] = S[((part * 9 + mu) * 3 + q) * NT + threadIdx.x];
                    Ub[c12_lidx(g, mu, parity ^ 1, q, sb[mu])] = S[((part * 9 + 4 + mu) * 3 + q) * NT + threadIdx.x];
                }
#pragma unroll
            for (int q = 0; q < 3; ++q) Wb[c12_gidx(g, parity, q, s)] = S[((part * 9 + 8) * 3 + q) * NT + threadIdx.x];
        }
    }
    if (ACC) warp_partial(rsum, bt.partial);
    {
        const int w = __reduce_add_sync(0xffffffffu, fb);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&bt.state[f].fallbacks, w);
    }
}

// R over all links of each field from the double-float storage (same block
// map as the half-sweep: kDFThreads sites per block).
__global__ void __launch_bounds__(kDFThreads) k_functional_df(SweepBatch bt) {
    const int f = field_of_block(bt.desc, bt.nf, blockIdx.x);
    const FieldDesc fd = bt.desc[f];
    const Geom g = fd.geo;
    const int s = (blockIdx.x - fd.blk0) * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (s < g.vh) {
        const float4* __restrict__ Uh = reinterpret_cast<const float4*>(fd.U);
        const float4* __restrict__ Ul = reinterpret_cast<const float4*>(fd.Ulo);
        float sh = 0.f, sl = 0.f;
#pragma unroll 1
        for (int p = 0; p < 2; ++p)
#pragma unroll 1
            for (int mu = 0; mu < 4; ++mu) {
                DC m[6];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float4 h = Uh[c12_lidx(g, mu, p, q, s)], l = Ul[c12_lidx(g, mu, p, q, s)];
                    m[2 * q] = DC{make_float2(h.x, l.x), make_float2(h.y, l.y)};
                    m[2 * q + 1] = DC{make_float2(h.z, l.z), make_float2(h.w, l.w)};
                }
                const DC r22 = dc_row2(m, 2);
                float th = m[0].re.x, tl = m[0].re.y, uh = m[0].im.x, ul = m[0].im.y;
                dd_add(th, tl, m[4].re);
                dd_add(th, tl, r22.re);
                dd_add(uh, ul, m[4].im);
                dd_add(uh, ul, r22.im);
                const float2 tr = dd_norm(th, tl), ti = dd_norm(uh, ul);
                dd_mac(sh, sl, tr, tr);
                dd_mac(sh, sl, ti, ti);
            }
        r = (double)sh + (double)sl;
    }
    warp_partial(r, bt.partial);
}

// FP64 full layout -> double-float compact storage (rows 0 and 1): hi =
// fl32(x), lo = fl32(x - hi), for nmat matrices per site and parity.
__global__ void __launch_bounds__(256) k_to_df(const cplx<double>* __restrict__ src, float4* __restrict__ hi,
                                               float4* __restrict__ lo, Geom g, int nmat, int nfields) {
    const long long per_field = 2LL * nmat * g.vh;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= per_field * nfields) return;
    const int f = (int)(id / per_field);
    const int r = (int)(id - (long long)f * per_field);
    const int mp = r / g.vh, s = r - mp * g.vh;
    const cplx<double>* sf = src + (size_t)f * 18 * nmat * g.vh + (size_t)mp * 9 * g.vh + s;
    const size_t o = (size_t)f * 6 * nmat * g.vh + (size_t)mp * 3 * g.vh + s;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const cplx<double> a = sf[(size_t)(2 * q) * g.vh], b = sf[(size_t)(2 * q + 1) * g.vh];
        const float2 ar = dd_from_double(a.x), ai = dd_from_double(a.y), br = dd_from_double(b.x),
                     bi = dd_from_double(b.y);
        hi[o + (size_t)q * g.vh] = make_float4(ar.x, ai.x, br.x, bi.x);
        lo[o + (size_t)q * g.vh] = make_float4(ar.y, ai.y, br.y, bi.y);
    }
}

// identity transform in double-float compact storage
__global__ void __launch_bounds__(256) k_identity_df(float4* __restrict__ hi, float4* __restrict__ lo, Geom g,
                                                     int nfields) {
    const long long n = 2LL * g.vh * nfields;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int f = (int)(id / (2LL * g.vh));
    const int r = (int)(id - (long long)f * 2 * g.vh);
    const int p = r / g.vh, s = r - p * g.vh;
    const size_t o = (size_t)f * 6 * g.vh + (size_t)p * 3 * g.vh + s;
    // rows 0, 1 of 1: (1, 0), (0, 0) | (0, 0), (0, 0) | (1, 0), (0, 0)
    hi[o] = make_float4(1.f, 0.f, 0.f, 0.f);
    hi[o + g.vh] = make_float4(0.f, 0.f, 0.f, 0.f);
    hi[o + 2 * (size_t)g.vh] = make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 3; ++q) lo[o + (size_t)q * g.vh] = make_float4(0.f, 0.f, 0.f, 0.f);
}

static size_t halfsweep_smem_df() { return sizeof(float4) * 54 * kDFThreads; }

int df_threads() { return kDFThreads; }

int prepare_halfsweep_df() {
    const int smem = (int)halfsweep_smem_df();
    MCG_CK(cudaFuncSetAttribute(k_halfsweep_df<false, kDFThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MCG_CK(cudaFuncSetAttribute(k_halfsweep_df<true, kDFThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return 0;
}

void launch_halfsweep_df(bool acc, const SweepBatch& bt, int parity, int nblocks, cudaStream_t st) {
    const size_t smem = halfsweep_smem_df();
    if (acc)
        k_halfsweep_df<true, kDFThreads><<<nblocks, kDFThreads, smem, st>>>(bt, parity);
    else
        k_halfsweep_df<false, kDFThreads><<<nblocks, kDFThreads, smem, st>>>(bt, parity);
}

void launch_functional_df(const SweepBatch& bt, int nblocks, cudaStream_t st) {
    k_functional_df<<<nblocks, kDFThreads, 0, st>>>(bt);
}

static unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

int launch_to_df(const double* src, void* hi, void* lo, const Geom& g, int nmat, int nfields, cudaStream_t st) {
    const long long n = 2LL * nmat * g.vh * nfields;
    k_to_df<<<blocks_of(n), 256, 0, st>>>((const cplx<double>*)src, (float4*)hi, (float4*)lo, g, nmat, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

int launch_identity_df(void* hi, void* lo, const Geom& g, int nfields, cudaStream_t st) {
    const long long n = 2LL * g.vh * nfields;
    k_identity_df<<<blocks_of(n), 256, 0, st>>>((float4*)hi, (float4*)lo, g, nfields);
    MCG_CK(cudaGetLastError());
    note_launches(1);
    return 0;
}

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_sweep_df)

}  // namespace mcg
