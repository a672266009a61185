// The FP32 MCG half-sweep on the compact working storage (the FP32 sweeps of
// the mixed-precision schedule and FP32 fields): kernel, launch and set-up.
#include <cuda_runtime.h>

#include "mcg_common.cuh"
#include "mcg_internal.h"
#include "mcg_sweep.cuh"

namespace mcg {

// ---------------------------------------------------------------------------
// FP32 half-sweep on the compact storage: one thread per site, the site's
// nine matrices (forward links U_mu(x), backward links U_mu(x - mu), W(x)) as
// their rows 0 and 1: the forward links in registers (48 floats), the
// backward links and W in shared memory; the three subgroup steps unrolled
// with compile-time indices.  Row-2 entries are rebuilt where a step needs
// them; G acting on rows (P, 2) of a forward link changes row P only in the
// stored part (row 2 stays implied), and M G^dag acts on each row of a
// backward link separately.
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
// compact forward links m[0..3] (registers), the compact backward links and
// the transform W in shared memory (wst: 3 chunks per thread).  Returns 1 if
// the local solve left the Newton path.
template <int P, int Q, int R, int NT>
__device__ __forceinline__ int c12_subgroup_step(cplx<float> (&m)[4][6], float4* bst, float4* wst,
                                                 const float omega) {
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
    // the transform: rows P, Q of G W (kept in shared memory between the
    // steps, so no subgroup element stays live in registers)
    {
        cplx<float> w[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 v = wst[q * NT + threadIdx.x];
            w[2 * q] = mk(v.x, v.y);
            w[2 * q + 1] = mk(v.z, v.w);
        }
        c12_left_update_pk<P, Q>(w, G);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            wst[q * NT + threadIdx.x] = make_float4(w[2 * q].x, w[2 * q].y, w[2 * q + 1].x, w[2 * q + 1].y);
    }
    asm volatile("" ::: "memory");
    return fb;
}

// One thread per site.  The 4 forward links are loaded straight into
// registers (12 16-byte loads in flight); the 4 backward links and W are
// staged into shared memory by cp.async meanwhile.  The backward links and W
// are read and written there by each subgroup step.  Keeping half of the
// site's state out of registers removes most spills at the 168-register
// budget of 3 blocks of 128 threads per SM (W in shared memory: +3 % inside a
// fix over keeping the three subgroup elements for a final update of W).
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

        const float omega = (float)fd.omega;
        fb += c12_subgroup_step<0, 1, 2, NT>(m, bst, wstage, omega);
        fb += c12_subgroup_step<0, 2, 1, NT>(m, bst, wstage, omega);
        fb += c12_subgroup_step<1, 2, 0, NT>(m, bst, wstage, omega);

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

// dynamic shared memory: the staged W and backward links (15 chunks per
// thread: 30 KB for 128 threads)
static size_t halfsweep_smem_c12(int nt) { return sizeof(float4) * 15 * nt; }

template <typename K>
static int raise_smem_c12(K kernel, size_t smem) {
    MCG_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return 0;
}

int prepare_halfsweep_c12(int nt) {
    const size_t smem = halfsweep_smem_c12(nt);
    int rc = 0;
    if (nt == 256) {
        if ((rc = raise_smem_c12(k_halfsweep_c12<false, 256, 1>, smem)) ||
            (rc = raise_smem_c12(k_halfsweep_c12<true, 256, 1>, smem)))
            return rc;
    } else if (nt == 128) {
        if ((rc = raise_smem_c12(k_halfsweep_c12<false, 128, 3>, smem)) ||
            (rc = raise_smem_c12(k_halfsweep_c12<true, 128, 3>, smem)))
            return rc;
    } else {
        if ((rc = raise_smem_c12(k_halfsweep_c12<false, 64, 6>, smem)) ||
            (rc = raise_smem_c12(k_halfsweep_c12<true, 64, 6>, smem)))
            return rc;
    }
    return 0;
}

// Occupancy: the register file holds 3 blocks of 128 threads (<= 168
// registers per thread).
void launch_halfsweep_c12(int nt, bool acc, const SweepBatch& bt, int parity, int nblocks, cudaStream_t st) {
    const size_t smem = halfsweep_smem_c12(nt);
    if (nt == 256) {
        if (acc)
            k_halfsweep_c12<true, 256, 1><<<nblocks, 256, smem, st>>>(bt, parity);
        else
            k_halfsweep_c12<false, 256, 1><<<nblocks, 256, smem, st>>>(bt, parity);
    } else if (nt == 128) {
        if (acc)
            k_halfsweep_c12<true, 128, 3><<<nblocks, 128, smem, st>>>(bt, parity);
        else
            k_halfsweep_c12<false, 128, 3><<<nblocks, 128, smem, st>>>(bt, parity);
    } else {
        if (acc)
            k_halfsweep_c12<true, 64, 6><<<nblocks, 64, smem, st>>>(bt, parity);
        else
            k_halfsweep_c12<false, 64, 6><<<nblocks, 64, smem, st>>>(bt, parity);
    }
}

// index-check counter of this unit (MCG_CHECK builds)
MCG_BOUND_READER(bound_hits_sweep_f32)

}  // namespace mcg
