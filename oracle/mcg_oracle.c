/*
 * FP64 CPU oracle for Maximal Center Gauge (MCG) fixing with stout and
 * over-improved stout preconditioning (O Cais, Kamleh, Langfeld, Lasscock,
 * Leinweber, Moran, Sternbeck, von Smekal 2008).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or table with the CUDA path: it is a plain, slow, sequential-per-site
 * restatement of what the method computes, written for reading against the
 * paper.  Every loop over sites may run under OpenMP; results do not depend on
 * the thread count (same-parity site updates touch disjoint links, reductions
 * sum fixed chunks in index order).
 *
 * Layout (canonical host layout): site index i = x + Nx*(y + Ny*(z + Nz*t)),
 *   U[(i*4 + mu)*9 + 3*row + col]   complex double, mu = 0..3 is x,y,z,t
 *   G[i*9 + 3*row + col]            complex double (gauge transform Omega(x))
 *   m[i*4 + mu]                     int8 center sector in {-1, 0, +1}
 *
 * Readings where the paper is silent (each stated where it is used):
 *   - the site update maximises the local functional exactly over the three
 *     SU(2) subgroups (0,1), (0,2), (1,2) in that order, one hit each,
 *     even sites then odd sites;
 *   - the stop rule is V_U(k) - V_U(k-1) < tol on the normalised functional;
 *   - links and Omega are re-unitarised every reunit_every sweeps;
 *   - stout smearing is isotropic in 4D and updates all links at once.
 *   - simulated annealing (named in Sec. III.B as a way to higher maxima, not
 *     specified): Metropolis hits on the same subgroup moves, proposals and
 *     acceptances drawn from Philox4x64-10 with a counter per (site, sweep,
 *     subgroup and hit, field), temperatures given per sweep (orc_anneal).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NCHUNK 256 /* fixed reduction chunking: result independent of threads */

/* ------------------------------------------------------------------ */
/* lattice geometry                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
    int n[4];
    long vol;
} geom;

static geom make_geom(const int* dims) {
    geom g;
    for (int d = 0; d < 4; ++d) g.n[d] = dims[d];
    g.vol = (long)dims[0] * dims[1] * dims[2] * dims[3];
    return g;
}

static void coords_of(const geom* g, long i, int* c) {
    for (int d = 0; d < 4; ++d) {
        c[d] = (int)(i % g->n[d]);
        i /= g->n[d];
    }
}

static long index_of(const geom* g, const int* c) {
    return c[0] + (long)g->n[0] * (c[1] + (long)g->n[1] * (c[2] + (long)g->n[2] * c[3]));
}

/* site i displaced by `step` lattice units along direction mu, periodic */
static long shift(const geom* g, long i, int mu, int step) {
    int c[4];
    coords_of(g, i, c);
    c[mu] = ((c[mu] + step) % g->n[mu] + g->n[mu]) % g->n[mu];
    return index_of(g, c);
}

static int parity_of(const geom* g, long i) {
    int c[4];
    coords_of(g, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* ------------------------------------------------------------------ */
/* 3x3 complex matrices                                                 */
/* ------------------------------------------------------------------ */
static void m_mul(cplx* r, const cplx* a, const cplx* b) { /* r = a b */
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(r, t, sizeof t);
}

static void m_mul_nd(cplx* r, const cplx* a, const cplx* b) { /* r = a b^dag */
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * conj(b[3 * j + k]);
            t[3 * i + j] = s;
        }
    memcpy(r, t, sizeof t);
}

static void m_mul_dn(cplx* r, const cplx* a, const cplx* b) { /* r = a^dag b */
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += conj(a[3 * k + i]) * b[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(r, t, sizeof t);
}

static void m_dag(cplx* r, const cplx* a) {
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[3 * i + j] = conj(a[3 * j + i]);
    memcpy(r, t, sizeof t);
}

static cplx m_trace(const cplx* a) { return (a[0] + a[4]) + a[8]; }

static void m_set_identity(cplx* a) {
    for (int k = 0; k < 9; ++k) a[k] = 0;
    a[0] = a[4] = a[8] = 1;
}

static double m_fnorm(const cplx* a) {
    double s = 0;
    for (int k = 0; k < 9; ++k) s += creal(a[k] * conj(a[k]));
    return sqrt(s);
}

/* Project a near-SU(3) matrix back onto SU(3): normalise row 0; remove its
 * component from row 1 and normalise; row 2 = conj(row0 x row1). */
static void m_reunitarise(cplx* a) {
    cplx* r0 = a;
    cplx* r1 = a + 3;
    cplx* r2 = a + 6;
    double n0 = sqrt(creal(r0[0] * conj(r0[0]) + r0[1] * conj(r0[1]) + r0[2] * conj(r0[2])));
    for (int k = 0; k < 3; ++k) r0[k] /= n0;
    cplx p = conj(r0[0]) * r1[0] + conj(r0[1]) * r1[1] + conj(r0[2]) * r1[2];
    for (int k = 0; k < 3; ++k) r1[k] -= p * r0[k];
    double n1 = sqrt(creal(r1[0] * conj(r1[0]) + r1[1] * conj(r1[1]) + r1[2] * conj(r1[2])));
    for (int k = 0; k < 3; ++k) r1[k] /= n1;
    r2[0] = conj(r0[1] * r1[2] - r0[2] * r1[1]);
    r2[1] = conj(r0[2] * r1[0] - r0[0] * r1[2]);
    r2[2] = conj(r0[0] * r1[1] - r0[1] * r1[0]);
}

static inline cplx* link(cplx* U, long i, int mu) { return U + (i * 4 + mu) * 9; }
static inline const cplx* clink(const cplx* U, long i, int mu) { return U + (i * 4 + mu) * 9; }

/* ------------------------------------------------------------------ */
/* Observables                                                          */
/* ------------------------------------------------------------------ */

/* Gauge functional R = sum_{x,mu} |tr U_mu(x)|^2; V_U = R / (9 * 4V)
 * (Sec. II.A, the MCG condition V_U[Omega]). */
double orc_functional_R(const int* dims, const cplx* U) {
    geom g = make_geom(dims);
    long nl = g.vol * 4;
    double part[NCHUNK];
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < NCHUNK; ++ch) {
        long lo = nl * ch / NCHUNK, hi = nl * (ch + 1) / NCHUNK;
        double s = 0;
        for (long l = lo; l < hi; ++l) {
            cplx t = m_trace(U + l * 9);
            s += creal(t) * creal(t) + cimag(t) * cimag(t);
        }
        part[ch] = s;
    }
    double r = 0;
    for (int ch = 0; ch < NCHUNK; ++ch) r += part[ch];
    return r;
}

/* Mean plaquette <(1/3) Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag>
 * over the 6V plaquettes; gauge invariant (Sec. III.A). */
double orc_plaquette(const int* dims, const cplx* U) {
    geom g = make_geom(dims);
    double part[NCHUNK];
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < NCHUNK; ++ch) {
        long lo = g.vol * ch / NCHUNK, hi = g.vol * (ch + 1) / NCHUNK;
        double s = 0;
        for (long i = lo; i < hi; ++i)
            for (int mu = 0; mu < 4; ++mu)
                for (int nu = mu + 1; nu < 4; ++nu) {
                    cplx a[9], b[9];
                    m_mul(a, clink(U, i, mu), clink(U, shift(&g, i, mu, 1), nu));
                    m_mul_nd(b, a, clink(U, shift(&g, i, nu, 1), mu));
                    m_mul_nd(a, b, clink(U, i, nu));
                    s += creal(m_trace(a)) / 3.0;
                }
        part[ch] = s;
    }
    double r = 0;
    for (int ch = 0; ch < NCHUNK; ++ch) r += part[ch];
    return r / (6.0 * (double)g.vol);
}

/* U_mu(x) <- Omega(x) U_mu(x) Omega(x+mu)^dag, in place (Sec. II.A/II.B:
 * the gauge-transformed field U^Omega). */
void orc_apply_gauge(const int* dims, cplx* U, const cplx* G) {
    geom g = make_geom(dims);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < g.vol; ++i)
        for (int mu = 0; mu < 4; ++mu) {
            cplx t[9];
            m_mul(t, G + i * 9, link(U, i, mu));
            m_mul_nd(link(U, i, mu), t, G + shift(&g, i, mu, 1) * 9);
        }
}

void orc_reunitarise_field(long nmat, cplx* M) {
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nmat; ++k) m_reunitarise(M + k * 9);
}

/* Omega_out(x) = Omega_b(x) Omega_a(x), composition of two transforms. */
void orc_compose_gauge(long vol, const cplx* Gb, const cplx* Ga, cplx* Gout) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < vol; ++i) m_mul(Gout + i * 9, Gb + i * 9, Ga + i * 9);
}

/* ------------------------------------------------------------------ */
/* Local SU(2)-subgroup maximisation                                    */
/* ------------------------------------------------------------------ */

/* Cyclic Jacobi diagonalisation of a symmetric 4x4 matrix: A = V diag(al) V^T,
 * columns of V are eigenvectors.  Runs until the off-diagonal norm is below
 * 1e-15 of the Frobenius norm (or 60 sweeps). */
static void jacobi4(const double* Ain, double* V, double* al) {
    double A[4][4];
    double fro = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            A[i][j] = 0.5 * (Ain[4 * i + j] + Ain[4 * j + i]);
            fro += A[i][j] * A[i][j];
            V[4 * i + j] = (i == j) ? 1.0 : 0.0;
        }
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += 2 * A[p][q] * A[p][q];
        if (sqrt(off) <= 1e-15 * fro || off == 0) break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0) continue;
                /* rotation angle that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < 4; ++k) { /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) { /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) { /* V <- V J */
                    double vkp = V[4 * k + p], vkq = V[4 * k + q];
                    V[4 * k + p] = c * vkp - s * vkq;
                    V[4 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 4; ++i) al[i] = A[i][i];
}

/*
 * Maximise F(a) = a^T A a + 2 b^T a over the unit sphere |a| = 1 in R^4
 * (A symmetric 4x4 row-major, b in R^4).  The global maximiser satisfies
 * (mu I - A) a = b with mu >= alpha_max (the trust-region optimality
 * condition).  Easy case: mu is the root right of alpha_max of
 * ||a(mu)|| = 1, a(mu) = sum_i beta_i / (mu - alpha_i) v_i, beta_i = v_i . b.
 * It is solved for the offset d = mu - alpha_max, with the gaps
 * alpha_max - alpha_i formed once, so that d keeps full relative precision
 * when it is tiny (beta_top, the component of b in the top eigenspace, near
 * zero): Newton on 1/||a|| - 1 (Moré and Sorensen), which is concave and
 * increasing in d and so climbs monotonically to the root from any point
 * with ||a|| >= 1, inside the bracket [|beta_top|, ||b||] with bisection as a
 * safeguard.  When the weights off the top eigenspace alone give ||a|| >= 1
 * at d = 0 the root lies beyond the root of their equation, which is solved
 * first the same way and starts the full iteration.
 * Hard case (b has no component along the top eigenspace and the rest of the
 * solution has norm < 1): mu = alpha_max and a = partial + t v_max with t > 0
 * after fixing the sign of v_max so that its largest-magnitude component is
 * positive.  The paper is silent on this degenerate case; several maximisers
 * are equally correct there.
 * Returns 0 (easy case) or 1 (hard case); a is normalised to |a| = 1.
 */
int orc_trs_solve(const double* A, const double* b, double* a) {
    double V[16], al[4];
    jacobi4(A, V, al);
    double scale = 0;
    for (int i = 0; i < 4; ++i) scale = fmax(scale, fabs(al[i]));
    double bn = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
    scale = fmax(scale, bn);
    if (scale == 0) { /* F constant on the sphere: keep the identity */
        a[0] = 1; a[1] = a[2] = a[3] = 0;
        return 1;
    }
    int imax = 0;
    for (int i = 1; i < 4; ++i)
        if (al[i] > al[imax]) imax = i;
    double amax = al[imax];
    double beta[4];
    for (int i = 0; i < 4; ++i)
        beta[i] = V[0 * 4 + i] * b[0] + V[1 * 4 + i] * b[1] + V[2 * 4 + i] * b[2] + V[3 * 4 + i] * b[3];

    /* top eigenspace: eigenvalues within 1e-13*scale of the largest */
    int top[4];
    double btop = 0;
    for (int i = 0; i < 4; ++i) {
        top[i] = (amax - al[i]) <= 1e-13 * scale;
        if (top[i]) btop += beta[i] * beta[i];
    }
    btop = sqrt(btop);
    if (btop <= 1e-14 * scale) {
        double pn2 = 0, coef[4];
        for (int i = 0; i < 4; ++i) {
            coef[i] = top[i] ? 0.0 : beta[i] / (amax - al[i]);
            pn2 += coef[i] * coef[i];
        }
        if (pn2 < 1.0) {
            double vm[4];
            for (int k = 0; k < 4; ++k) vm[k] = V[4 * k + imax];
            int kbig = 0;
            for (int k = 1; k < 4; ++k)
                if (fabs(vm[k]) > fabs(vm[kbig])) kbig = k;
            double sgn = vm[kbig] >= 0 ? 1.0 : -1.0;
            double t = sqrt(1.0 - pn2);
            for (int k = 0; k < 4; ++k) {
                double s = 0;
                for (int i = 0; i < 4; ++i) s += V[4 * k + i] * coef[i];
                a[k] = s + t * sgn * vm[k];
            }
            double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
            for (int k = 0; k < 4; ++k) a[k] /= an;
            return 1;
        }
    }

    /* gaps to the largest eigenvalue (0 on the top eigenspace) and the norm
     * of the solution without the top weights at d = 0 */
    double gap[4], rest2 = 0;
    for (int i = 0; i < 4; ++i) {
        gap[i] = top[i] ? 0.0 : amax - al[i];
        if (!top[i]) rest2 += beta[i] * beta[i] / (gap[i] * gap[i]);
    }
    /* bracket: ||a|| >= btop / d, so d = btop lies left of the root;
     * ||a|| <= ||b|| / d, so d = ||b|| lies right of it */
    double lo = btop, hi = bn, d = btop;
    if (rest2 >= 1.0) {
        double dr = 0;
        for (int it = 0; it < 200; ++it) {
            double s2 = 0, s3 = 0;
            for (int i = 0; i < 4; ++i) {
                if (top[i]) continue;
                double e = dr + gap[i];
                double q = beta[i] * beta[i] / (e * e);
                s2 += q;
                s3 += q / e;
            }
            if (!(s3 > 0)) break;
            double step = (sqrt(s2) - 1.0) * s2 / s3;
            dr += step;
            if (!(step > 1e-15 * dr)) break;
        }
        if (dr > d) d = fmin(dr, hi);
    }
    for (int it = 0; it < 200; ++it) {
        double s2 = 0, s3 = 0;
        for (int i = 0; i < 4; ++i) {
            if (beta[i] == 0.0) continue; /* a zero weight contributes nothing, also where d + gap is 0 */
            double e = d + gap[i];
            double q = beta[i] * beta[i] / (e * e);
            s2 += q;
            s3 += q / e;
        }
        double n = sqrt(s2);
        if (n >= 1.0) lo = fmax(lo, d);
        else hi = fmin(hi, d);
        double next = d + (n - 1.0) * s2 / s3; /* Newton on 1/n - 1 */
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (next == d || fabs(next - d) <= 1e-15 * d) {
            d = next;
            break;
        }
        d = next;
        if (hi - lo <= 4e-16 * d) break;
    }
    double an2 = 0;
    for (int k = 0; k < 4; ++k) {
        double s = 0;
        for (int i = 0; i < 4; ++i)
            if (beta[i] != 0.0) s += V[4 * k + i] * beta[i] / (d + gap[i]);
        a[k] = s;
        an2 += s * s;
    }
    double an = sqrt(an2);
    for (int k = 0; k < 4; ++k) a[k] /= an;
    return 0;
}

/* Coefficients of tr(G M) as an affine function of the SU(2) parameter a,
 * for G the subgroup (p,q) embedding of g = a0 + i a.sigma:
 *   tr(G M) = M_rr + sum_k w_k a_k,
 *   w = (m11 + m22, i(m21 + m12), m21 - m12, i(m11 - m22)),
 * with m the (p,q) block of M.  For a backward link B (which becomes B G^dag)
 * tr(B G^dag) = tr(G^dag B) takes the same form with a_1..a_3 negated. */
static void subgroup_coeffs(const cplx* M, int p, int q, int r, int backward, cplx* c, cplx* w) {
    cplx m11 = M[3 * p + p], m12 = M[3 * p + q], m21 = M[3 * q + p], m22 = M[3 * q + q];
    *c = M[3 * r + r];
    w[0] = m11 + m22;
    w[1] = I * (m21 + m12);
    w[2] = m21 - m12;
    w[3] = I * (m11 - m22);
    if (backward) {
        w[1] = -w[1];
        w[2] = -w[2];
        w[3] = -w[3];
    }
}

/* One site update at x: for (p,q) = (0,1), (0,2), (1,2), choose the SU(2)
 * subgroup element G maximising sum over the 8 links at x of |tr|^2, then
 * U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dag, Omega(x) <- G Omega(x).
 * Returns the number of hard-case solves. */
static int site_update(const geom* g, cplx* U, cplx* Om, long x, double omega) {
    static const int PQ[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};
    int hard = 0;
    cplx* F[4];
    cplx* B[4];
    for (int mu = 0; mu < 4; ++mu) {
        F[mu] = link(U, x, mu);
        B[mu] = link(U, shift(g, x, mu, -1), mu);
    }
    for (int s = 0; s < 3; ++s) {
        int p = PQ[s][0], q = PQ[s][1], r = PQ[s][2];
        double A[16] = {0}, b[4] = {0};
        for (int l = 0; l < 8; ++l) {
            cplx c, w[4];
            subgroup_coeffs(l < 4 ? F[l] : B[l - 4], p, q, r, l >= 4, &c, w);
            for (int k = 0; k < 4; ++k) {
                b[k] += creal(conj(c) * w[k]);
                for (int j = 0; j < 4; ++j) A[4 * k + j] += creal(conj(w[k]) * w[j]);
            }
        }
        double a[4];
        hard += orc_trs_solve(A, b, a);
        if (omega != 1.0) {
            /* over-relaxation: a -> normalise((1 - omega) e0 + omega a), the
             * truncated form of g^omega (not part of the paper's method) */
            a[0] = (1.0 - omega) + omega * a[0];
            for (int k = 1; k < 4; ++k) a[k] *= omega;
            double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
            for (int k = 0; k < 4; ++k) a[k] /= an;
        }
        cplx g11 = a[0] + I * a[3], g12 = a[2] + I * a[1];
        cplx g21 = -a[2] + I * a[1], g22 = a[0] - I * a[3];
        for (int mu = 0; mu < 4; ++mu) {
            cplx* f = F[mu];
            for (int k = 0; k < 3; ++k) { /* rows p, q of G F */
                cplx xp = f[3 * p + k], xq = f[3 * q + k];
                f[3 * p + k] = g11 * xp + g12 * xq;
                f[3 * q + k] = g21 * xp + g22 * xq;
            }
            cplx* bb = B[mu];
            for (int k = 0; k < 3; ++k) { /* columns p, q of B G^dag */
                cplx xp = bb[3 * k + p], xq = bb[3 * k + q];
                bb[3 * k + p] = xp * conj(g11) + xq * conj(g12);
                bb[3 * k + q] = xp * conj(g21) + xq * conj(g22);
            }
        }
        cplx* o = Om + x * 9;
        for (int k = 0; k < 3; ++k) {
            cplx xp = o[3 * p + k], xq = o[3 * q + k];
            o[3 * p + k] = g11 * xp + g12 * xq;
            o[3 * q + k] = g21 * xp + g22 * xq;
        }
    }
    return hard;
}

/* Update every site of one parity (0: x+y+z+t even).  Same-parity sites share
 * no link, so the order within the parity does not matter.  Returns the number
 * of hard-case local solves. */
long orc_halfsweep(const int* dims, cplx* U, cplx* Om, int parity, double omega) {
    geom g = make_geom(dims);
    long hard = 0;
#pragma omp parallel for schedule(static) reduction(+ : hard)
    for (long x = 0; x < g.vol; ++x)
        if (parity_of(&g, x) == parity) hard += site_update(&g, U, Om, x, omega);
    return hard;
}

/*
 * MCG relaxation (Sec. II.A, II.B): full sweeps (even then odd half-sweep)
 * until V_U(k) - V_U(k-1) < tol or max_sweeps, where V_U = R / (9 * 4V).
 * Every reunit_every sweeps (if > 0) links and Omega are re-unitarised.
 * omega = 1 is the plain relaxation; omega != 1 over-relaxes each subgroup
 * step (an optional accelerator, not described in the paper).
 * R_hist[0..sweeps] receives R before the first sweep and after each sweep.
 * Returns 0 if converged, 1 if max_sweeps was reached.
 */
/* The half-sweep of one t-slab of a larger lattice (the lattice split into
 * slabs along t, one per process).  `dims` is the local array: the slab's
 * layers at local t in [t_lo, t_hi) plus ghost layers outside that range,
 * which hold the links owned by the neighbouring slabs that the slab's sites
 * touch (the backward t-links of its first layer).  Updates the sites with
 * t_lo <= t < t_hi whose parity on the whole lattice,
 * (x + y + z + t + t_offset) mod 2, equals `parity`, with the site update of
 * orc_halfsweep; ghost links are read and written like any other.  Same-parity
 * sites share no link, so slabs updated one after another (or at once, each
 * on its own copy with the ghosts exchanged around the call) give exactly the
 * half-sweep of the whole lattice. */
long orc_halfsweep_slab(const int* dims, cplx* U, cplx* Om, int parity, double omega, int t_lo, int t_hi,
                        int t_offset) {
    geom g = make_geom(dims);
    long hard = 0;
#pragma omp parallel for schedule(static) reduction(+ : hard)
    for (long x = 0; x < g.vol; ++x) {
        int c[4];
        coords_of(&g, x, c);
        if (c[3] < t_lo || c[3] >= t_hi) continue;
        if (((c[0] + c[1] + c[2] + c[3] + t_offset) & 1) != parity) continue;
        hard += site_update(&g, U, Om, x, omega);
    }
    return hard;
}

int orc_fix(const int* dims, cplx* U, cplx* Om, double tol, int max_sweeps, int reunit_every, double omega,
            double* R_hist, int* sweeps_out, long* hard_out) {
    geom g = make_geom(dims);
    double norm = 1.0 / (9.0 * 4.0 * (double)g.vol);
    double Rprev = orc_functional_R(dims, U);
    if (R_hist) R_hist[0] = Rprev;
    long hard = 0;
    int k;
    for (k = 1; k <= max_sweeps; ++k) {
        hard += orc_halfsweep(dims, U, Om, 0, omega);
        hard += orc_halfsweep(dims, U, Om, 1, omega);
        if (reunit_every > 0 && k % reunit_every == 0) {
            orc_reunitarise_field(g.vol * 4, U);
            orc_reunitarise_field(g.vol, Om);
        }
        double R = orc_functional_R(dims, U);
        if (R_hist) R_hist[k] = R;
        if ((R - Rprev) * norm < tol) {
            *sweeps_out = k;
            if (hard_out) *hard_out = hard;
            return 0;
        }
        Rprev = R;
    }
    *sweeps_out = max_sweeps;
    if (hard_out) *hard_out = hard;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Simulated annealing of the gauge transform (Sec. III.B: the SU(2) route  */
/* to higher maxima, here for the SU(3) functional as a Gribov-copy     */
/* search variant ahead of the relaxation)                              */
/* ------------------------------------------------------------------ */

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds on the counter (c0, c1, c2, c3) with
 * key (k0, k1); each round maps
 *   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * hi / lo the halves of the 128-bit product, and the key advances by the
 * Weyl increments (W0, W1) between rounds. */
void orc_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* 64 random bits -> a double in [0, 1): the top 53 bits times 2^-53 (exact). */
static double unit_interval(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }

/* Sum over the 8 links at x of |tr|^2 (the site's share of R). */
static double site_functional(cplx* const* F, cplx* const* B) {
    double s = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        cplx tf = m_trace(F[mu]), tb = m_trace(B[mu]);
        s += creal(tf) * creal(tf) + cimag(tf) * cimag(tf);
        s += creal(tb) * creal(tb) + cimag(tb) * cimag(tb);
    }
    return s;
}

/*
 * One annealing site update at x, temperature T.  For the subgroups (0,1),
 * (0,2), (1,2) in turn, nhit Metropolis hits: the counter
 * (x, sweep, subgroup * nhit + hit, field) under key (seed, 0) gives four
 * words w0..w3; the proposal is the SU(2) element a = (a0, v) with
 * v_k = eps (2 u(w_{k-1}) - 1), a0 = sqrt(1 - |v|^2) (its law is even under
 * a -> a^dag, so the Metropolis rule keeps exp(F/T) times Haar measure
 * invariant), embedded as G in rows/columns (p, q); the move
 * U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dag, Omega(x) <- G Omega(x)
 * changes the site functional by dF, and is accepted when dF >= 0 or
 * u(w3) < exp(dF / T).  Returns the number of accepted hits.
 */
static long anneal_site(const geom* g, cplx* U, cplx* Om, long x, double T, long sweep, int nhit, double eps,
                        uint64_t seed, uint64_t field) {
    static const int PQ[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};
    cplx* F[4];
    cplx* B[4];
    for (int mu = 0; mu < 4; ++mu) {
        F[mu] = link(U, x, mu);
        B[mu] = link(U, shift(g, x, mu, -1), mu);
    }
    const uint64_t key[2] = {seed, 0};
    long accepted = 0;
    for (int s = 0; s < 3; ++s) {
        int p = PQ[s][0], q = PQ[s][1], r = PQ[s][2];
        for (int h = 0; h < nhit; ++h) {
            uint64_t ctr[4] = {(uint64_t)x, (uint64_t)sweep, (uint64_t)(s * nhit + h), field}, w[4];
            orc_philox4x64(ctr, key, w);
            double v1 = eps * (2.0 * unit_interval(w[0]) - 1.0);
            double v2 = eps * (2.0 * unit_interval(w[1]) - 1.0);
            double v3 = eps * (2.0 * unit_interval(w[2]) - 1.0);
            double a0 = sqrt(1.0 - (v1 * v1 + v2 * v2 + v3 * v3));
            cplx G[9] = {0};
            G[3 * r + r] = 1.0;
            G[3 * p + p] = a0 + I * v3;
            G[3 * p + q] = v2 + I * v1;
            G[3 * q + p] = -v2 + I * v1;
            G[3 * q + q] = a0 - I * v3;
            cplx Fn[4][9], Bn[4][9];
            for (int mu = 0; mu < 4; ++mu) {
                m_mul(Fn[mu], G, F[mu]);
                m_mul_nd(Bn[mu], B[mu], G);
            }
            cplx* Fp[4] = {Fn[0], Fn[1], Fn[2], Fn[3]};
            cplx* Bp[4] = {Bn[0], Bn[1], Bn[2], Bn[3]};
            double dF = site_functional(Fp, Bp) - site_functional(F, B);
            if (dF >= 0.0 || unit_interval(w[3]) < exp(dF / T)) {
                for (int mu = 0; mu < 4; ++mu) {
                    memcpy(F[mu], Fn[mu], sizeof(Fn[mu]));
                    memcpy(B[mu], Bn[mu], sizeof(Bn[mu]));
                }
                cplx o[9];
                m_mul(o, G, Om + x * 9);
                memcpy(Om + x * 9, o, sizeof(o));
                ++accepted;
            }
        }
    }
    return accepted;
}

/* Annealing update of every site of one parity at temperature T (sweep
 * number `sweep` in the random-number counter).  Returns accepted hits. */
long orc_anneal_halfsweep(const int* dims, cplx* U, cplx* Om, int parity, double T, long sweep, int nhit, double eps,
                          uint64_t seed, uint64_t field) {
    geom g = make_geom(dims);
    long acc = 0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (long x = 0; x < g.vol; ++x)
        if (parity_of(&g, x) == parity) acc += anneal_site(&g, U, Om, x, T, sweep, nhit, eps, seed, field);
    return acc;
}

/*
 * Simulated annealing: for k = 0 .. nsweeps-1, an even then an odd annealing
 * half-sweep at temperature T[k] with sweep number first_sweep + k; then
 * links and Omega are re-unitarised once.  Returns the accepted hits.
 */
long orc_anneal(const int* dims, cplx* U, cplx* Om, const double* T, int nsweeps, long first_sweep, int nhit,
                double eps, uint64_t seed, uint64_t field) {
    geom g = make_geom(dims);
    long acc = 0;
    for (int k = 0; k < nsweeps; ++k) {
        acc += orc_anneal_halfsweep(dims, U, Om, 0, T[k], first_sweep + k, nhit, eps, seed, field);
        acc += orc_anneal_halfsweep(dims, U, Om, 1, T[k], first_sweep + k, nhit, eps, seed, field);
    }
    orc_reunitarise_field(g.vol * 4, U);
    orc_reunitarise_field(g.vol, Om);
    return acc;
}

/* ------------------------------------------------------------------ */
/* Stout and over-improved stout smearing                               */
/* ------------------------------------------------------------------ */

/* exp(X) for a 3x3 complex X by Taylor series with scaling and squaring:
 * X / 2^s has Frobenius norm <= 1/4, the series runs until a term falls below
 * 1e-18, then the result is squared s times. */
void orc_expm(const cplx* X, cplx* E) {
    double nrm = m_fnorm(X);
    int s = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        ++s;
    }
    double sc = ldexp(1.0, -s);
    cplx Y[9], term[9], t2[9];
    for (int k = 0; k < 9; ++k) Y[k] = X[k] * sc;
    m_set_identity(E);
    m_set_identity(term);
    for (int n = 1; n < 40; ++n) {
        m_mul(t2, term, Y);
        for (int k = 0; k < 9; ++k) term[k] = t2[k] / (double)n;
        for (int k = 0; k < 9; ++k) E[k] += term[k];
        if (m_fnorm(term) < 1e-18) break;
    }
    for (int j = 0; j < s; ++j) m_mul(E, E, E);
}

/* Staple sum of U_mu(x) with plaquette weight cp and rectangle weight cr:
 * cp * (2 plaquette staples per nu) + cr * (6 rectangle staples per nu:
 * two 1x2 with the link on the short side, four 2x1 with the link on a long
 * side), summed over nu != mu.  Every staple is a path from x to x+mu. */
static void staple_sum(const geom* g, const cplx* U, long x, int mu, double cp, double cr, cplx* C) {
    for (int k = 0; k < 9; ++k) C[k] = 0;
    long xpm = shift(g, x, mu, 1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        cplx a[9], b[9];
        long xpn = shift(g, x, nu, 1), xmn = shift(g, x, nu, -1);
        long xmn_pm = shift(g, xmn, mu, 1);
        /* upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag */
        m_mul(a, clink(U, x, nu), clink(U, xpn, mu));
        m_mul_nd(b, a, clink(U, xpm, nu));
        for (int k = 0; k < 9; ++k) C[k] += cp * b[k];
        /* lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) */
        m_mul_dn(a, clink(U, xmn, nu), clink(U, xmn, mu));
        m_mul(b, a, clink(U, xmn_pm, nu));
        for (int k = 0; k < 9; ++k) C[k] += cp * b[k];
        if (cr == 0) continue;
        long xp2n = shift(g, xpn, nu, 1), xm2n = shift(g, xmn, nu, -1);
        long xmm = shift(g, x, mu, -1);
        cplx r[9];
        /* 1x2 up: U_nu(x) U_nu(x+nu) U_mu(x+2nu) U_nu(x+mu+nu)^dag U_nu(x+mu)^dag */
        m_mul(a, clink(U, x, nu), clink(U, xpn, nu));
        m_mul(b, a, clink(U, xp2n, mu));
        m_mul_nd(a, b, clink(U, shift(g, xpm, nu, 1), nu));
        m_mul_nd(r, a, clink(U, xpm, nu));
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
        /* 1x2 down: U_nu(x-nu)^dag U_nu(x-2nu)^dag U_mu(x-2nu) U_nu(x-2nu+mu) U_nu(x-nu+mu) */
        {
            /* (U_nu(x-2nu) U_nu(x-nu))^dag = U_nu(x-nu)^dag U_nu(x-2nu)^dag */
            cplx p2[9];
            m_mul(p2, clink(U, xm2n, nu), clink(U, xmn, nu));
            m_dag(a, p2);
        }
        m_mul(b, a, clink(U, xm2n, mu));
        m_mul(a, b, clink(U, shift(g, xm2n, mu, 1), nu));
        m_mul(r, a, clink(U, xmn_pm, nu));
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
        /* 2x1 forward up: U_nu(x) U_mu(x+nu) U_mu(x+nu+mu) U_nu(x+2mu)^dag U_mu(x+mu)^dag */
        long xp2m = shift(g, xpm, mu, 1);
        m_mul(a, clink(U, x, nu), clink(U, xpn, mu));
        m_mul(b, a, clink(U, shift(g, xpn, mu, 1), mu));
        m_mul_nd(a, b, clink(U, xp2m, nu));
        m_mul_nd(r, a, clink(U, xpm, mu));
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
        /* 2x1 forward down: U_nu(x-nu)^dag U_mu(x-nu) U_mu(x-nu+mu) U_nu(x-nu+2mu) U_mu(x+mu)^dag */
        m_mul_dn(a, clink(U, xmn, nu), clink(U, xmn, mu));
        m_mul(b, a, clink(U, xmn_pm, mu));
        m_mul(a, b, clink(U, shift(g, xmn_pm, mu, 1), nu));
        m_mul_nd(r, a, clink(U, xpm, mu));
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
        /* 2x1 backward up: U_mu(x-mu)^dag U_nu(x-mu) U_mu(x-mu+nu) U_mu(x+nu) U_nu(x+mu)^dag */
        m_mul_dn(a, clink(U, xmm, mu), clink(U, xmm, nu));
        m_mul(b, a, clink(U, shift(g, xmm, nu, 1), mu));
        m_mul(a, b, clink(U, xpn, mu));
        m_mul_nd(r, a, clink(U, xpm, nu));
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
        /* 2x1 backward down: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_mu(x-nu) U_nu(x-nu+mu) */
        {
            long xmm_mn = shift(g, xmm, nu, -1);
            cplx p2[9];
            m_mul(p2, clink(U, xmm_mn, nu), clink(U, xmm, mu)); /* U_nu(x-mu-nu) U_mu(x-mu) */
            m_dag(a, p2);                                         /* U_mu(x-mu)^dag U_nu(x-mu-nu)^dag */
            m_mul(b, a, clink(U, xmm_mn, mu));
            m_mul(a, b, clink(U, xmn, mu));
            m_mul(r, a, clink(U, xmn_pm, nu));
        }
        for (int k = 0; k < 9; ++k) C[k] += cr * r[k];
    }
}

/*
 * One smearing step, all links at once from the old field:
 *   C_mu(x) = rho * S_mu(x),  Om = C_mu(x) U_mu(x)^dag,
 *   Q = (i/2)(Om^dag - Om) - (i/6) tr(Om^dag - Om),  U' = exp(iQ) U.
 * S is the staple sum of the over-improved action with weights
 * (5 - 2 eps)/3 on plaquette staples and -(1 - eps)/12 on rectangle staples;
 * eps = 1 is plain stout smearing (weights 1 and 0).  (Sec. II.B: stout and
 * over-improved stout smearing as cited there.)
 */
void orc_smear_step(const int* dims, const cplx* Uin, cplx* Uout, double rho, double eps) {
    geom g = make_geom(dims);
    double cp = (5.0 - 2.0 * eps) / 3.0;
    double cr = -(1.0 - eps) / 12.0;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g.vol; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            cplx C[9], Om[9], Q[9], X[9], E[9];
            staple_sum(&g, Uin, x, mu, cp, cr, C);
            for (int k = 0; k < 9; ++k) C[k] *= rho;
            m_mul_nd(Om, C, clink(Uin, x, mu));
            cplx tr = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx d = conj(Om[3 * j + i]) - Om[3 * i + j]; /* (Om^dag - Om)_ij */
                    Q[3 * i + j] = 0.5 * I * d;
                    if (i == j) tr += d;
                }
            for (int i = 0; i < 3; ++i) Q[4 * i] -= (I / 6.0) * tr;
            for (int k = 0; k < 9; ++k) X[k] = I * Q[k];
            orc_expm(X, E);
            m_mul(link(Uout, x, mu), E, clink(Uin, x, mu));
        }
}

void orc_smear(const int* dims, const cplx* Uin, cplx* Uout, double rho, double eps, int nsteps) {
    geom g = make_geom(dims);
    size_t bytes = (size_t)g.vol * 4 * 9 * sizeof(cplx);
    if (nsteps <= 0) {
        memcpy(Uout, Uin, bytes);
        return;
    }
    cplx* tmp = (cplx*)malloc(bytes);
    const cplx* src = Uin;
    for (int s = 0; s < nsteps; ++s) {
        /* ping-pong so that the last step writes Uout */
        cplx* dst = ((nsteps - 1 - s) % 2 == 0) ? Uout : tmp;
        orc_smear_step(dims, src, dst, rho, eps);
        src = dst;
    }
    free(tmp);
}

/* ------------------------------------------------------------------ */
/* Center projection and P-vortices                                     */
/* ------------------------------------------------------------------ */

/* Center sector of a link (Sec. II.A): the phase of tr U nearest to
 * 2 pi m / 3, m in {-1, 0, +1}.  Decided by exact comparisons:
 *   m = 0  if Re t >= 0 and |Im t| <= sqrt(3) Re t   (|phi| <= pi/3),
 *   m = +1 else if Im t >= 0                         (pi/3 < phi <= pi),
 *   m = -1 otherwise.
 * t = (U00 + U11) + U22.  This is also the center element Z closest to U on
 * the group manifold, since Re tr(Z^dag U) = |t| cos(phi - 2 pi m / 3). */
void orc_center_project(const int* dims, const cplx* U, int8_t* m) {
    geom g = make_geom(dims);
    const double sqrt3 = 1.7320508075688772;
#pragma omp parallel for schedule(static)
    for (long l = 0; l < g.vol * 4; ++l) {
        const cplx* u = U + l * 9;
        double re = (creal(u[0]) + creal(u[4])) + creal(u[8]);
        double im = (cimag(u[0]) + cimag(u[4])) + cimag(u[8]);
        volatile double lim = sqrt3 * re; /* a plain product, never fused */
        int8_t s;
        if (re >= 0 && fabs(im) <= lim) s = 0;
        else if (im >= 0) s = 1;
        else s = -1;
        m[l] = s;
    }
}

/* Count P-vortices (Sec. II.A): a plaquette is pierced when the product of its
 * four center links is non-trivial, i.e. when
 * (m_mu(x) + m_nu(x+mu) - m_mu(x+nu) - m_nu(x)) mod 3 != 0.
 * per_plane[6] (may be NULL) receives the count for planes 01,02,03,12,13,23.
 * Returns the total. */
long long orc_vortex_count(const int* dims, const int8_t* m, long long* per_plane) {
    geom g = make_geom(dims);
    long long cnt[6] = {0};
    for (long x = 0; x < g.vol; ++x) {
        int pl = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
                int n = m[x * 4 + mu] + m[shift(&g, x, mu, 1) * 4 + nu] - m[shift(&g, x, nu, 1) * 4 + mu] -
                        m[x * 4 + nu];
                if (((n % 3) + 3) % 3 != 0) cnt[pl]++;
            }
    }
    long long tot = 0;
    for (int p = 0; p < 6; ++p) {
        if (per_plane) per_plane[p] = cnt[p];
        tot += cnt[p];
    }
    return tot;
}

/* ------------------------------------------------------------------ */
/* Vortex removal, the vortex-only field and Wilson loops (Sec. III.A)   */
/* ------------------------------------------------------------------ */

/* The center element exp(2 pi i m / 3) of sector m as (cos, sin); the
 * values for m = +-1 are the literals -1/2 and +-sqrt(3)/2. */
static void center_phase(int m, double* c, double* s) {
    if (m == 0) {
        *c = 1.0;
        *s = 0.0;
    } else {
        *c = -0.5;
        *s = m > 0 ? 0.8660254037844386 : -0.8660254037844386;
    }
}

/* Vortex-removed field U'_mu(x) = Z_mu(x)^dag U_mu(x), Z the center element
 * of the link's sector m (Sec. III.A): every entry u becomes conj(Z) u, i.e.
 * re' = c re + s im, im' = c im - s re (products and sums written out, never
 * fused). */
void orc_vortex_remove(const int* dims, const cplx* U, const int8_t* m, cplx* Uout) {
    geom g = make_geom(dims);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < g.vol * 4; ++l) {
        double c, sn;
        center_phase(m[l], &c, &sn);
        for (int e = 0; e < 9; ++e) {
            const double re = creal(U[l * 9 + e]), im = cimag(U[l * 9 + e]);
            volatile double a = c * re, b = sn * im, d = c * im, f = sn * re;
            Uout[l * 9 + e] = (a + b) + I * (d - f);
        }
    }
}

/* The vortex-only field: Z_mu(x) = exp(2 pi i m_mu(x) / 3) times the identity. */
void orc_center_links(const int* dims, const int8_t* m, cplx* Z) {
    geom g = make_geom(dims);
    for (long l = 0; l < g.vol * 4; ++l) {
        double c, sn;
        center_phase(m[l], &c, &sn);
        for (int e = 0; e < 9; ++e) Z[l * 9 + e] = (e % 4 == 0) ? c + I * sn : 0;
    }
}

/* product of L links along mu from site x: U_mu(x) U_mu(x+mu) ... */
static void line_product(const geom* g, const cplx* U, long x, int mu, int L, cplx* out) {
    m_set_identity(out);
    cplx t[9];
    long y = x;
    for (int k = 0; k < L; ++k) {
        m_mul(t, out, clink(U, y, mu));
        memcpy(out, t, sizeof t);
        y = shift(g, y, mu, 1);
    }
}

/* Planar Wilson loops W(R, T) (Sec. III.A): R links along a spatial axis i
 * in {x, y, z}, T links along t (mu = 3), averaged over all V translations
 * and the three spatial axes,
 *   W(R,T) = < (1/3) Re tr [ S_i^R(x) S_t^T(x + R i) S_i^R(x + T t)^dag S_t^T(x)^dag ] >,
 * S_mu^L(x) the product of L links along mu from x.  out[(R-1)*Tmax + T-1]
 * for 1 <= R <= Rmax, 1 <= T <= Tmax; sums in fixed chunks. */
void orc_wilson_loops(const int* dims, const cplx* U, int Rmax, int Tmax, double* out) {
    geom g = make_geom(dims);
    const int npair = Rmax * Tmax;
    double* part = calloc((size_t)NCHUNK * npair, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < NCHUNK; ++ch) {
        const long x0 = g.vol * ch / NCHUNK, x1 = g.vol * (ch + 1) / NCHUNK;
        for (long x = x0; x < x1; ++x)
            for (int i = 0; i < 3; ++i)
                for (int R = 1; R <= Rmax; ++R) {
                    cplx S[9], A[9], B[9], C[9], D[9], t1[9], t2[9];
                    line_product(&g, U, x, i, R, S);
                    long xr = x;
                    for (int k = 0; k < R; ++k) xr = shift(&g, xr, i, 1);
                    for (int T = 1; T <= Tmax; ++T) {
                        long xt = x;
                        for (int k = 0; k < T; ++k) xt = shift(&g, xt, 3, 1);
                        line_product(&g, U, xr, 3, T, A);  /* S_t^T(x + R i) */
                        line_product(&g, U, xt, i, R, B);  /* S_i^R(x + T t) */
                        line_product(&g, U, x, 3, T, C);   /* S_t^T(x)       */
                        m_mul(t1, S, A);
                        m_mul_nd(t2, t1, B);
                        m_mul_nd(D, t2, C);
                        part[(size_t)ch * npair + (R - 1) * Tmax + (T - 1)] += creal(m_trace(D)) / 3.0;
                    }
                }
    }
    for (int k = 0; k < npair; ++k) {
        double acc = 0;
        for (int ch = 0; ch < NCHUNK; ++ch) acc += part[(size_t)ch * npair + k];
        out[k] = acc / (3.0 * g.vol);
    }
    free(part);
}

/* Off-axis spatial paths (Sec. III.A mentions off-axis loops without
 * fixing the paths; reading): the path from x to x + r, r = (r0, r1, r2),
 * takes L = |r0| + |r1| + |r2| unit steps; step k (1-based) goes along the
 * axis j with the largest deficit k |r_j| / L - n_j (n_j: steps taken along j
 * so far), ties to the lowest j, in the direction of sign(r_j).  For an
 * on-axis r this is the straight path.  Writes the axes (0..2) and signs of
 * the L steps; returns L. */
static int path_steps(const int* r, int* axis, int* sign) {
    const int L = abs(r[0]) + abs(r[1]) + abs(r[2]);
    int n[3] = {0, 0, 0};
    for (int k = 1; k <= L; ++k) {
        int best = -1;
        double bd = -1e300;
        for (int j = 0; j < 3; ++j) {
            if (n[j] >= abs(r[j])) continue;
            const double d = (double)k * abs(r[j]) / L - n[j];
            if (d > bd) {
                bd = d;
                best = j;
            }
        }
        axis[k - 1] = best;
        sign[k - 1] = r[best] > 0 ? 1 : -1;
        n[best]++;
    }
    return L;
}

/* product of the links along the path of r from x (backward steps use
 * U_j(y - j)^dag) */
static void path_product(const geom* g, const cplx* U, long x, const int* r, cplx* out) {
    int axis[64], sign[64];
    const int L = path_steps(r, axis, sign);
    m_set_identity(out);
    cplx t[9], d[9];
    long y = x;
    for (int k = 0; k < L; ++k) {
        if (sign[k] > 0) {
            m_mul(t, out, clink(U, y, axis[k]));
            y = shift(g, y, axis[k], 1);
        } else {
            y = shift(g, y, axis[k], -1);
            m_dag(d, clink(U, y, axis[k]));
            m_mul(t, out, d);
        }
        memcpy(out, t, sizeof t);
    }
}

/* the distinct images of r under axis permutations and sign flips */
static int cubic_images(const int* r, int img[48][3]) {
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int n = 0;
    for (int p = 0; p < 6; ++p)
        for (int sgn = 0; sgn < 8; ++sgn) {
            int v[3];
            for (int j = 0; j < 3; ++j) v[j] = r[perm[p][j]] * ((sgn >> j) & 1 ? -1 : 1);
            int dup = 0;
            for (int q = 0; q < n && !dup; ++q) dup = img[q][0] == v[0] && img[q][1] == v[1] && img[q][2] == v[2];
            if (!dup) {
                img[n][0] = v[0];
                img[n][1] = v[1];
                img[n][2] = v[2];
                ++n;
            }
        }
    return n;
}

/* Wilson loops with off-axis spatial sides (Sec. III.A): for each vector
 * r of vecs (nvec x 3) and 1 <= T <= Tmax, the mean over all translations x
 * and all distinct cubic images r' of r of
 *   (1/3) Re tr [ P_r'(x) S_t^T(x + r') P_r'(x + T t)^dag S_t^T(x)^dag ],
 * P the path product above.  out[v * Tmax + T - 1]; sums in fixed chunks. */
void orc_wilson_loops_offaxis(const int* dims, const cplx* U, const int* vecs, int nvec, int Tmax, double* out) {
    geom g = make_geom(dims);
    for (int v = 0; v < nvec; ++v) {
        int img[48][3];
        const int ni = cubic_images(vecs + 3 * v, img);
        double* part = calloc((size_t)NCHUNK * Tmax, sizeof(double));
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < NCHUNK; ++ch) {
            const long x0 = g.vol * ch / NCHUNK, x1 = g.vol * (ch + 1) / NCHUNK;
            for (long x = x0; x < x1; ++x)
                for (int q = 0; q < ni; ++q) {
                    cplx P[9], A[9], B[9], C[9], t1[9], t2[9], D[9];
                    path_product(&g, U, x, img[q], P);
                    long xr = x;
                    for (int j = 0; j < 3; ++j) {
                        for (int k = 0; k < abs(img[q][j]); ++k) xr = shift(&g, xr, j, img[q][j] > 0 ? 1 : -1);
                    }
                    for (int T = 1; T <= Tmax; ++T) {
                        long xt = x;
                        for (int k = 0; k < T; ++k) xt = shift(&g, xt, 3, 1);
                        line_product(&g, U, xr, 3, T, A);
                        path_product(&g, U, xt, img[q], B);
                        line_product(&g, U, x, 3, T, C);
                        m_mul(t1, P, A);
                        m_mul_nd(t2, t1, B);
                        m_mul_nd(D, t2, C);
                        part[(size_t)ch * Tmax + (T - 1)] += creal(m_trace(D)) / 3.0;
                    }
                }
        }
        for (int T = 0; T < Tmax; ++T) {
            double acc = 0;
            for (int ch = 0; ch < NCHUNK; ++ch) acc += part[(size_t)ch * Tmax + T];
            out[v * Tmax + T] = acc / ((double)ni * g.vol);
        }
        free(part);
    }
}

/* ------------------------------------------------------------------ */
/* Gradient of R with respect to the gauge transform                    */
/* ------------------------------------------------------------------ */

/* The eight SU(3) generators T_a = lambda_a / 2 (Gell-Mann matrices,
 * tr(lambda_a lambda_b) = 2 delta_ab), row-major 3x3. */
static void gell_mann_half(cplx T[8][9]) {
    for (int a = 0; a < 8; ++a)
        for (int k = 0; k < 9; ++k) T[a][k] = 0;
    T[0][1] = T[0][3] = 0.5;
    T[1][1] = -0.5 * I;
    T[1][3] = 0.5 * I;
    T[2][0] = 0.5;
    T[2][4] = -0.5;
    T[3][2] = T[3][6] = 0.5;
    T[4][2] = -0.5 * I;
    T[4][6] = 0.5 * I;
    T[5][5] = T[5][7] = 0.5;
    T[6][5] = -0.5 * I;
    T[6][7] = 0.5 * I;
    T[7][0] = T[7][4] = 0.5 / sqrt(3.0);
    T[7][8] = -1.0 / sqrt(3.0);
}

void orc_generators(cplx* out) {
    cplx T[8][9];
    gell_mann_half(T);
    memcpy(out, T, sizeof T);
}

/* d R / d eps_a at eps = 0 for Omega(x) -> exp(i eps T_a) Omega(x):
 * U_mu(x) -> (1 + i eps T_a) U_mu(x) and U_mu(x-mu) -> U_mu(x-mu)(1 - i eps T_a),
 * so with t_f = tr U_mu(x), t_b = tr U_mu(x-mu):
 *   dR_a(x) = sum_mu 2 Re[conj(t_f) i tr(T_a U_mu(x))]
 *           + 2 Re[conj(t_b) (-i) tr(T_a U_mu(x-mu))].
 * grad is V x 8. */
void orc_grad_R(const int* dims, const cplx* U, double* grad) {
    geom g = make_geom(dims);
    cplx T[8][9];
    gell_mann_half(T);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g.vol; ++x) {
        for (int a = 0; a < 8; ++a) grad[x * 8 + a] = 0;
        for (int mu = 0; mu < 4; ++mu) {
            const cplx* F = clink(U, x, mu);
            const cplx* B = clink(U, shift(&g, x, mu, -1), mu);
            cplx tf = m_trace(F), tb = m_trace(B);
            for (int a = 0; a < 8; ++a) {
                cplx t1[9], t2[9];
                m_mul(t1, T[a], F);
                m_mul(t2, T[a], B);
                grad[x * 8 + a] += 2.0 * creal(conj(tf) * I * m_trace(t1)) + 2.0 * creal(conj(tb) * (-I) * m_trace(t2));
            }
        }
    }
}


/* ------------------------------------------------------------------ */
/* Differentiation through stout / over-improved stout smearing         */
/* ------------------------------------------------------------------ */

/* n x n complex matrix exponential (Taylor + scaling and squaring), used on
 * the 6x6 block matrix of the Frechet identity below. */
static void expm_n(int n, const cplx* X, cplx* E) {
    double nrm = 0;
    for (int k = 0; k < n * n; ++k) nrm += creal(X[k] * conj(X[k]));
    nrm = sqrt(nrm);
    int s = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        ++s;
    }
    double sc = ldexp(1.0, -s);
    cplx Y[36], term[36], t2[36];
    for (int k = 0; k < n * n; ++k) Y[k] = X[k] * sc;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) E[n * i + j] = term[n * i + j] = (i == j) ? 1.0 : 0.0;
    for (int m = 1; m < 60; ++m) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                cplx acc = 0;
                for (int k = 0; k < n; ++k) acc += term[n * i + k] * Y[n * k + j];
                t2[n * i + j] = acc / (double)m;
            }
        double tn = 0;
        for (int k = 0; k < n * n; ++k) {
            term[k] = t2[k];
            E[k] += term[k];
            tn += creal(term[k] * conj(term[k]));
        }
        if (sqrt(tn) < 1e-18) break;
    }
    for (int r = 0; r < s; ++r) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                cplx acc = 0;
                for (int k = 0; k < n; ++k) acc += E[n * i + k] * E[n * k + j];
                t2[n * i + j] = acc;
            }
        for (int k = 0; k < n * n; ++k) E[k] = t2[k];
    }
}

/* Frechet derivative of exp at X in direction A, L(X, A) = d/dt exp(X + tA)
 * at t = 0, as the upper-right block of exp([[X, A], [0, X]]) (the block
 * triangular identity of Van Loan 1978 / Mathias 1996). */
void orc_expm_frechet(const cplx* X, const cplx* A, cplx* L) {
    cplx M[36], E[36];
    for (int k = 0; k < 36; ++k) M[k] = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            M[6 * i + j] = X[3 * i + j];
            M[6 * (i + 3) + (j + 3)] = X[3 * i + j];
            M[6 * i + (j + 3)] = A[3 * i + j];
        }
    expm_n(6, M, E);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) L[3 * i + j] = E[6 * i + (j + 3)];
}

/* One staple as a path of links from x to x+mu: factor k is U_dir(site) or
 * its dagger. */
typedef struct {
    int n;
    long site[5];
    int dir[5];
    int dag[5];
    double w;
} staple_path;

static int add_path(staple_path* P, int np, double w, int n, const long* site, const int* dir, const int* dag) {
    P[np].n = n;
    P[np].w = w;
    for (int k = 0; k < n; ++k) {
        P[np].site[k] = site[k];
        P[np].dir[k] = dir[k];
        P[np].dag[k] = dag[k];
    }
    return np + 1;
}

/* The staples of U_mu(x) entering the smearing step, as paths with their
 * weights: per nu != mu two plaquette staples (weight cp) and, if cr != 0,
 * six rectangle staples (weight cr), the same set as staple_sum(). */
static int staple_paths(const geom* g, long x, int mu, double cp, double cr, staple_path* P) {
    int np = 0;
    long xpm = shift(g, x, mu, 1), xmm = shift(g, x, mu, -1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long xpn = shift(g, x, nu, 1), xmn = shift(g, x, nu, -1);
        long xmn_pm = shift(g, xmn, mu, 1);
        {
            long s[3] = {x, xpn, xpm};
            int d[3] = {nu, mu, nu}, h[3] = {0, 0, 1};
            np = add_path(P, np, cp, 3, s, d, h);
        }
        {
            long s[3] = {xmn, xmn, xmn_pm};
            int d[3] = {nu, mu, nu}, h[3] = {1, 0, 0};
            np = add_path(P, np, cp, 3, s, d, h);
        }
        if (cr == 0) continue;
        long xp2n = shift(g, xpn, nu, 1), xm2n = shift(g, xmn, nu, -1);
        long xp2m = shift(g, xpm, mu, 1);
        {   /* 1x2 up */
            long s[5] = {x, xpn, xp2n, shift(g, xpm, nu, 1), xpm};
            int d[5] = {nu, nu, mu, nu, nu}, h[5] = {0, 0, 0, 1, 1};
            np = add_path(P, np, cr, 5, s, d, h);
        }
        {   /* 1x2 down */
            long s[5] = {xmn, xm2n, xm2n, shift(g, xm2n, mu, 1), xmn_pm};
            int d[5] = {nu, nu, mu, nu, nu}, h[5] = {1, 1, 0, 0, 0};
            np = add_path(P, np, cr, 5, s, d, h);
        }
        {   /* 2x1 forward up */
            long s[5] = {x, xpn, shift(g, xpn, mu, 1), xp2m, xpm};
            int d[5] = {nu, mu, mu, nu, mu}, h[5] = {0, 0, 0, 1, 1};
            np = add_path(P, np, cr, 5, s, d, h);
        }
        {   /* 2x1 forward down */
            long s[5] = {xmn, xmn, xmn_pm, shift(g, xmn_pm, mu, 1), xpm};
            int d[5] = {nu, mu, mu, nu, mu}, h[5] = {1, 0, 0, 0, 1};
            np = add_path(P, np, cr, 5, s, d, h);
        }
        {   /* 2x1 backward up */
            long s[5] = {xmm, xmm, shift(g, xmm, nu, 1), xpn, xpm};
            int d[5] = {mu, nu, mu, mu, nu}, h[5] = {1, 0, 0, 0, 1};
            np = add_path(P, np, cr, 5, s, d, h);
        }
        {   /* 2x1 backward down */
            long xmm_mn = shift(g, xmm, nu, -1);
            long s[5] = {xmm, xmm_mn, xmm_mn, xmn, xmn_pm};
            int d[5] = {mu, nu, mu, mu, nu}, h[5] = {1, 1, 0, 0, 0};
            np = add_path(P, np, cr, 5, s, d, h);
        }
    }
    return np;
}

static void factor(const cplx* U, const staple_path* p, int k, cplx* out) {
    const cplx* m = clink(U, p->site[k], p->dir[k]);
    if (p->dag[k])
        m_dag(out, m);
    else
        memcpy(out, m, 9 * sizeof(cplx));
}

/* Staple sum rebuilt from the path list (for checking staple_paths against
 * staple_sum). */
void orc_staple_sum_paths(const int* dims, const cplx* U, long x, int mu, double cp, double cr, cplx* C) {
    geom g = make_geom(dims);
    staple_path P[24];
    int np = staple_paths(&g, x, mu, cp, cr, P);
    for (int k = 0; k < 9; ++k) C[k] = 0;
    for (int s = 0; s < np; ++s) {
        cplx W[9], f[9];
        factor(U, &P[s], 0, W);
        for (int k = 1; k < P[s].n; ++k) {
            factor(U, &P[s], k, f);
            m_mul(W, W, f);
        }
        for (int k = 0; k < 9; ++k) C[k] += P[s].w * W[k];
    }
}

void orc_staple_sum(const int* dims, const cplx* U, long x, int mu, double cp, double cr, cplx* C) {
    geom g = make_geom(dims);
    staple_sum(&g, U, x, mu, cp, cr, C);
}

/*
 * Reverse-mode derivative of one smearing step U' = exp(iQ(U)) U.
 * Gout holds the matrix gradient of a real loss with respect to U'
 * (Gout = dL/dRe U' + i dL/dIm U', so that dL = Re tr(Gout^dag dU')); Gin
 * receives the gradient with respect to U.  Chain rule, per link:
 *   direct:     Gin += exp(iQ)^dag Gout
 *   exp:        B = L(iQ, U Gout^dag)  (Frechet adjoint: tr(A L(X,E)) = tr(L(X,A) E))
 *   projection: K = (B - B^dag)/2 - tr((B - B^dag)/2)/3   (from Q's definition)
 *   Omega = C U^dag:  Gin += K C,  and Re tr(rho U^dag K dS) is scattered
 *               over every factor of every staple of the link.
 */
void orc_smear_step_backward(const int* dims, const cplx* U, const cplx* Gout, cplx* Gin, double rho, double eps) {
    geom g = make_geom(dims);
    const double cp = (5.0 - 2.0 * eps) / 3.0, cr = -(1.0 - eps) / 12.0;
    long nl = g.vol * 4;
    for (long l = 0; l < nl * 9; ++l) Gin[l] = 0;
    for (long x = 0; x < g.vol; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            const cplx* u = clink(U, x, mu);
            const cplx* go = Gout + (x * 4 + mu) * 9;
            cplx C[9], Om[9], Q[9], X[9], E[9], t[9], B[9], K[9], Y[9];
            staple_sum(&g, U, x, mu, cp, cr, C);
            for (int k = 0; k < 9; ++k) C[k] *= rho;
            m_mul_nd(Om, C, u);
            cplx tr = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx d = conj(Om[3 * j + i]) - Om[3 * i + j];
                    Q[3 * i + j] = 0.5 * I * d;
                    if (i == j) tr += d;
                }
            for (int i = 0; i < 3; ++i) Q[4 * i] -= (I / 6.0) * tr;
            for (int k = 0; k < 9; ++k) X[k] = I * Q[k];
            orc_expm(X, E);
            cplx* gi = Gin + (x * 4 + mu) * 9;
            m_mul_dn(t, E, go); /* E^dag Gout */
            for (int k = 0; k < 9; ++k) gi[k] += t[k];
            m_mul_nd(t, u, go); /* U Gout^dag */
            orc_expm_frechet(X, t, B);
            cplx trk = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    K[3 * i + j] = 0.5 * (B[3 * i + j] - conj(B[3 * j + i]));
                    if (i == j) trk += K[3 * i + j];
                }
            for (int i = 0; i < 3; ++i) K[4 * i] -= trk / 3.0;
            m_mul(t, K, C); /* K C */
            for (int k = 0; k < 9; ++k) gi[k] += t[k];
            m_mul_dn(Y, u, K); /* U^dag K */
            for (int k = 0; k < 9; ++k) Y[k] *= rho;
            staple_path P[24];
            int np = staple_paths(&g, x, mu, cp, cr, P);
            for (int s = 0; s < np; ++s) {
                int n = P[s].n;
                cplx F[5][9];
                for (int k = 0; k < n; ++k) factor(U, &P[s], k, F[k]);
                for (int j = 0; j < n; ++j) {
                    /* Z = A_{j+1} ... A_n (w Y) A_1 ... A_{j-1} */
                    cplx Z[9];
                    m_set_identity(Z);
                    for (int k = j + 1; k < n; ++k) m_mul(Z, Z, F[k]);
                    m_mul(Z, Z, Y);
                    for (int k = 0; k < j; ++k) m_mul(Z, Z, F[k]);
                    for (int k = 0; k < 9; ++k) Z[k] *= P[s].w;
                    cplx* gt = Gin + (P[s].site[j] * 4 + P[s].dir[j]) * 9;
                    if (P[s].dag[j]) {
                        for (int k = 0; k < 9; ++k) gt[k] += Z[k];
                    } else {
                        cplx Zd[9];
                        m_dag(Zd, Z);
                        for (int k = 0; k < 9; ++k) gt[k] += Zd[k];
                    }
                }
            }
        }
}

/* Matrix gradient of R = sum |tr U|^2: G = 2 tr(U) 1 per link. */
void orc_functional_matrix_grad(const int* dims, const cplx* U, cplx* G) {
    geom g = make_geom(dims);
    for (long l = 0; l < g.vol * 4; ++l) {
        cplx t = m_trace(U + l * 9);
        for (int k = 0; k < 9; ++k) G[l * 9 + k] = 0;
        G[l * 9 + 0] = G[l * 9 + 4] = G[l * 9 + 8] = 2.0 * t;
    }
}

int orc_version(void) { return 1; }
