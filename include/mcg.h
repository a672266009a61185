/*
 * libmcg — Maximal Center Gauge (MCG) fixing of 4D SU(3) lattice gauge fields
 * with stout / over-improved stout preconditioning, Z3 center projection and
 * P-vortex counting, on one NVIDIA GB300 (sm_103a).
 *
 * Method: A. O Cais et al., "Preconditioning Maximal Center Gauge with Stout
 * Link Smearing in SU(3)" (2008).  Sec. II.A defines the MCG functional, the
 * center projection and P-vortices; Sec. II.B the preconditioning pipeline;
 * Sec. III the smearing parameters.
 *
 * CONVENTIONS (every entry point)
 *  - Pointers named U, G, Z, S, grad are DEVICE pointers to caller-owned
 *    memory; pointers named *_out, *_host or counts are HOST pointers.
 *  - Calls are asynchronous on `stream` unless they return scalars through
 *    host pointers, in which case they synchronise `stream` before returning.
 *    `stream` may be 0 (the legacy default stream).
 *  - Return value: MCG_OK (0) or an mcg_status code; the message of the last
 *    failure on the calling thread is mcg_last_error().  No C++ exception
 *    crosses this boundary.
 *  - The library allocates only internal scratch (device work buffers, pinned
 *    host staging), cached across calls and freed by mcg_release().
 *  - That scratch, and the streams on which the relaxation captures its CUDA
 *    graphs, belong to the device: calls for one device are made from one
 *    host thread at a time (calls for different devices may run in parallel).
 *
 * LAYOUT (device, "even/odd SoA"), for a lattice Nx x Ny x Nz x Nt with every
 * extent even and >= 2, V = Nx Ny Nz Nt, Vh = V / 2:
 *   site x = (x,y,z,t), lexicographic index i = x + Nx (y + Ny (z + Nz t)),
 *   parity p = (x+y+z+t) mod 2, in-parity index s = i / 2;
 *   a complex number is (re, im) interleaved, in the field's precision;
 *   links  U_mu(x)[row][col]: complex element ((mu*2 + p)*9 + 3*row + col)*Vh + s
 *   gauge  Omega(x)[row][col]: complex element (p*9 + 3*row + col)*Vh + s
 *   center sector of U_mu(x): int8 element (mu*2 + p)*Vh + s, value in {-1,0,1}
 * A batch of `nfields` fields of the same dims is stored back to back
 * (field f starts at complex element f*72*Vh for links, f*18*Vh for gauge).
 * mu = 0,1,2,3 is the x,y,z,t direction.
 *
 * CANONICAL host layout (accepted by the pack/unpack calls): complex double
 * U[i][mu][row][col] and Omega[i][row][col], i lexicographic as above.
 */
#ifndef MCG_H
#define MCG_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCG_OK = 0,
    MCG_NOT_CONVERGED = 1, /* max_sweeps reached; results are valid          */
    MCG_BAD_DIMS = 2,      /* an extent is odd or < 2, or nfields < 1        */
    MCG_BAD_ARG = 3,       /* null pointer, aliasing, out-of-range parameter */
    MCG_BAD_INPUT = 4,     /* an input link or transform is not finite or   */
                           /* not in SU(3) (see "Input validation" below)   */
    MCG_CUDA_ERROR = 5     /* a CUDA runtime call failed                     */
} mcg_status;

typedef enum { MCG_F64 = 0, MCG_F32 = 1 } mcg_precision;

typedef struct {
    int dims[4];   /* Nx, Ny, Nz, Nt: each even and >= 2                        */
    int nfields;   /* fields of these dims stored back to back (>= 1)           */
    int precision; /* MCG_F64 or MCG_F32: element type of U / G arrays          */
} mcg_lattice;

/*
 * Parameters of the MCG relaxation (Sec. II.A).  The paper does not state its
 * stop rule (it counts blocks of 50 iterations); this library stops a field
 * at the first sweep k with V_U(k) - V_U(k-1) < tol, where
 * V_U = R / (9 * 4V), R = sum_{x,mu} |tr U_mu(x)|^2.
 */
typedef struct {
    double tol;        /* stop threshold on the per-sweep change of V_U (1e-10) */
    int max_sweeps;    /* upper bound on full sweeps (even + odd half-sweep)    */
    int check_every;   /* sweeps between host-side convergence polls (>= 1)     */
    int reunit_every;  /* FP64 sweeps: re-unitarise links and Omega every n     */
                       /* sweeps (0: off).  FP32 sweeps re-unitarise in FP32    */
                       /* every sweep inside the sweep kernel.                  */
    int fp32_sweeps;   /* MCG_F64 fields only: run up to this many sweeps in a  */
                       /* FP32 phase before the FP64 sweeps (0: plain FP64)     */
    double fp32_tol;   /* FP32 phase stops once its dV_U per sweep, averaged    */
    int fp32_window;   /* over the last fp32_window (1..31) sweeps, is below    */
                       /* fp32_tol (FP32 rounding makes single-sweep dV noisy)  */
    double fp32_overrelax; /* FP32 phase only: over-relaxation omega in (0,2); */
                       /* 1 = the plain relaxation.  Each subgroup step then    */
                       /* applies normalise((1-omega) + omega a) instead of a.  */
                       /* Not part of the paper's method; FP64 sweeps always    */
                       /* use the plain relaxation.                             */
    int fp64_solve32;  /* FP64 sweeps: 0 = the local 4x4 problem is solved to   */
                       /* FP64 precision (default); 1 = it is built and solved  */
                       /* in FP32 and only the solution is normalised and       */
                       /* applied in FP64 (G stays unitary, the field stays on  */
                       /* its gauge orbit, R and the stop rule stay FP64; each  */
                       /* site lands within ~1e-7 of its exact local maximum).  */
    int fp64_df;       /* FP64 sweeps: 1 = run them in double-float arithmetic */
                       /* (each real an FP32 pair hi + lo, ~48-bit significand, */
                       /* in the compact rows-0-and-1 storage; local problem  */
                       /* built and solved in FP32 as with fp64_solve32, its   */
                       /* solution normalised in FP64); R and the stop rule    */
                       /* stay FP64; the phase's transform is re-unitarised   */
                       /* in FP64 and applied to the FP64 links at the end, so */
                       /* the result is exactly on its gauge orbit.  GB300     */
                       /* runs FP64 at ~1/60 of its FP32 rate.  0 = FP64.      */
    int fp32_restart;  /* FP32 phase (MCG_F64 fields, fp32_sweeps > 0): a    */
                       /* field that has run this many sweeps                  */
                       /* since its last (re)start without reaching fp32_tol  */
                       /* restarts the phase from the call's input links and  */
                       /* the identity transform with the next              */
                       /* over-relaxation of omega - d, omega + d, omega - 2d, */
                       /* omega + 2d, ... (d = fp32_restart_domega; no restart */
                       /* once it leaves (0, 2)); its sweeps keep counting     */
                       /* toward fp32_sweeps.  0 = off.  Not part of the      */
                       /* paper's method: a way out of the slow, creeping     */
                       /* approach to a lower maximum that some over-relaxed  */
                       /* trajectories take.                                  */
    double fp32_restart_domega; /* >= 0 */
    int fp32_restart_random; /* 1: the k-th restart begins from a random gauge */
                       /* copy of the field it restarts from: the Haar-random */
                       /* transform W0 of mcg_random_gauge(seed =             */
                       /* MCG_RESTART_SEED, seq = k) is applied to the call's */
                       /* FP64 links and left-multiplies its transform G (the */
                       /* output stays U_out = G_out U_in).  0: from the same */
                       /* links.                                               */
    int fp32_restart_creep; /* FP32 phase: also restart (as above) a field that */
                       /* creeps: over the last fp32_restart_creep sweeps the  */
                       /* mean dV_U per sweep of every check_every chunk stayed */
                       /* within [2, 20] x fp32_tol and the last quarter of    */
                       /* those chunks averages more than half the first     */
                       /* quarter (no decay).  0 = off.                        */
    int fp32_plain_finish; /* 1: after the over-relaxed FP32 phase, plain    */
                       /* FP32 sweeps (omega = 1) until the same fp32_tol      */
                       /* criterion, before the hand-off: over-relaxation near */
                       /* a maximum leaves an oscillating residue that the     */
                       /* plain relaxation removes, cheaper in FP32 than in    */
                       /* the FP64-class phase.  0 = off.                      */
} mcg_params;

/* Seed of the random gauge copies of mcg_params.fp32_restart_random. */
#define MCG_RESTART_SEED 0x4D434752ull

/* One field of a heterogeneous batch: device pointers to its links and its
 * gauge transform (layout above) and its dims. */
typedef struct {
    void* U;
    void* G;
    int dims[4];
} mcg_field;

/* Per-field result of mcg_precondition_fix (Sec. II.B pipeline). */
typedef struct {
    double V_smeared;      /* V_U reached on the smeared field (0 if nsmear=0) */
    double V_fixed;        /* V_U reached on the preconditioned original field */
    double plaquette_in;   /* mean plaquette of the input field                */
    double plaquette_out;  /* mean plaquette of the final field (gauge inv.)   */
    long long vortices;    /* P-vortex plaquettes of the center projection     */
    double vortex_density; /* vortices / (6 V)                                  */
    int sweeps_smeared;    /* sweeps spent fixing the smeared field            */
    int sweeps_fixed;      /* sweeps spent fixing the preconditioned field     */
    int sweeps_fp32;       /* of those, sweeps run in the FP32 phase           */
    int status;            /* this field's (level's) fixes: MCG_OK when both    */
                           /* converged, else MCG_NOT_CONVERGED                 */
    int fp32_restarts;     /* restarts of the FP32 phase in this level's fixes */
                           /* (mcg_params.fp32_restart)                         */
} mcg_precond_result;

/*
 * Input validation.  mcg_smear, mcg_fix, mcg_anneal, mcg_precondition_fix,
 * mcg_precondition_levels, mcg_fix_batch and mcg_gribov_search first check,
 * in one pass over the caller's links (and transforms G where the call reads
 * them), that every matrix M is finite and in SU(3):
 * max_ij |(M M^dag - 1)_ij| <= tol and |det M - 1| <= tol, with tol = 1e-6 for
 * MCG_F64 fields and 1e-4 for MCG_F32 fields (far above rounding, far below a
 * real defect).  mcg_center_project checks finiteness only: the sector is a
 * function of tr U and is defined for any finite matrix.  On failure they
 * return MCG_BAD_INPUT before any other GPU work; mcg_last_error() names the
 * array and the first failing matrix (field, direction, parity, in-parity
 * site).  The check synchronises the stream.  (The paper works with SU(3)
 * fields, Sec. II.A; the check only refuses inputs outside that domain.)
 */

/* Library version (major*10000 + minor*100 + patch). */
int mcg_version(void);

/* Message describing the last failure on this thread ("" if none). */
const char* mcg_last_error(void);

/* Free all cached scratch (device and pinned host) and forget cached device
 * addresses.  Safe to call any time no libmcg call is in flight; later calls
 * re-create what they need. */
int mcg_release(void);

/* ---- layout conversion ---------------------------------------------------
 * Canonical (complex double, device) <-> even/odd SoA in lat->precision.
 * canon and U/G must not overlap. */
int mcg_pack_links(const double* canon, void* U, const mcg_lattice* lat, cudaStream_t stream);
int mcg_unpack_links(const void* U, double* canon, const mcg_lattice* lat, cudaStream_t stream);
int mcg_pack_gauge(const double* canon, void* G, const mcg_lattice* lat, cudaStream_t stream);
int mcg_unpack_gauge(const void* G, double* canon, const mcg_lattice* lat, cudaStream_t stream);
/* int8 center sectors, SoA -> canonical Z[i][mu]. */
int mcg_unpack_center(const int8_t* Z, int8_t* canon, const mcg_lattice* lat, cudaStream_t stream);

/* Element-wise precision conversion of n complex numbers (SoA to SoA, same
 * layout).  src_prec/dst_prec are mcg_precision values. */
int mcg_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t n_complex, cudaStream_t stream);

/* Omega(x) = 1 for every site. */
int mcg_set_identity_gauge(void* G, const mcg_lattice* lat, cudaStream_t stream);

/* ---- observables ---------------------------------------------------------- */

/* Mean plaquette <(1/3) Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag>
 * over 6V plaquettes, per field (Sec. III.A: gauge invariant).
 * out: host, nfields doubles.  Synchronises. */
int mcg_plaquette(const void* U, double* out, const mcg_lattice* lat, cudaStream_t stream);

/* MCG functional R = sum_{x,mu} |tr U_mu(x)|^2 per field (Sec. II.A; the
 * paper's V_U = R / (9 * 4V)).  R_out: host, nfields doubles.  Synchronises. */
int mcg_functional(const void* U, double* R_out, const mcg_lattice* lat, cudaStream_t stream);

/* ---- gauge transforms ----------------------------------------------------- */

/* U_mu(x) <- Omega(x) U_mu(x) Omega(x+mu)^dag in place (Sec. II.B: the
 * preconditioning transform applied to the original links). */
int mcg_apply_gauge(void* U, const void* G, const mcg_lattice* lat, cudaStream_t stream);

/* Project every link (which=0) or every Omega (which=1) back onto SU(3)
 * (Gram-Schmidt on rows 0,1; row 2 = conj(row0 x row1)); arithmetic in FP64. */
int mcg_reunitarise(void* M, int which, const mcg_lattice* lat, cudaStream_t stream);

/* ---- the method ----------------------------------------------------------- */

/*
 * n steps of stout smearing (eps = 1) or over-improved stout smearing
 * (Sec. II.B and III: stout rho = 0.1; over-improved rho = 0.06, eps = -0.25).
 * Each step updates all links at once from the old field:
 *   C_mu(x) = rho * [ (5-2eps)/3 * (plaquette staples) - (1-eps)/12 * (2x1 and
 *             1x2 rectangle staples) ],  Omega = C U^dag,
 *   Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega),  U' = exp(iQ) U.
 * U_in and U_out are fields of lat (U_out must not overlap U_in); n = 0 copies.
 * U_in is validated first (see "Input validation"; synchronises), then the
 * steps run asynchronously on `stream`.
 */
int mcg_smear(const void* U_in, void* U_out, const mcg_lattice* lat, double rho, double eps, int n,
              cudaStream_t stream);

/*
 * MCG relaxation (Sec. II.A; "as outlined in Langfeld 2003", not reproduced in
 * the paper): full sweeps = even then odd checkerboard half-sweep; each site
 * update picks, for the SU(2) subgroups (0,1), (0,2), (1,2) in turn, the
 * subgroup element G that exactly maximises sum over the 8 links at x of
 * |tr|^2, then U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dag and
 * Omega(x) <- G Omega(x).  In place on U and G (pass G = identity to start
 * fresh, or a random transform for a Gribov copy).  Per field, stops at the
 * first sweep with dV_U < params->tol, or at params->max_sweeps.
 * With lat->precision = MCG_F64 and params->fp32_sweeps > 0 the early sweeps
 * run in FP32 (links and the transform of this call in FP32, stored as rows 0
 * and 1 with row 2 implied by unitarity, R accumulated in FP64); the FP32
 * transform is then re-unitarised in FP64 and applied to the
 * FP64 links, which keeps them on the gauge orbit, and FP64 sweeps finish.
 * R_out (host, nfields, may be NULL): R after the last sweep.
 * sweeps_out (host, nfields, may be NULL): sweeps performed (FP32 + FP64).
 * R_hist (host, nfields x (max_sweeps+1), may be NULL): R before the first
 *   sweep and after each sweep (entries past the last sweep are 0).
 * Returns MCG_OK when every field converged, else MCG_NOT_CONVERGED.
 * Synchronises.
 */
int mcg_fix(void* U, void* G, const mcg_lattice* lat, const mcg_params* params, double* R_out,
            int* sweeps_out, double* R_hist, cudaStream_t stream);

/*
 * The local problem of one subgroup step of mcg_fix on its own, for n
 * problems at once (Sec. II.A: with the SU(2) element written a0 + i a.sigma,
 * |a| = 1, the site's share of R is a^T A a + 2 b.a + const; the step takes
 * the global maximum over the sphere).  A: DEVICE, n row-major 4x4 FP64
 * matrices (16 doubles each; only the upper triangle, column >= row, is read,
 * A is taken symmetric).  b: DEVICE, n x 4 FP64.  a_out: DEVICE, n x 4 FP64,
 * the maximisers.  fallback_out: DEVICE, n ints, or NULL: 1 where the solve
 * left the warm-started Newton path for the Jacobi + secular one.
 * precision MCG_F32: the solve of the FP32 and double-float sweeps (A and b
 * rounded to FP32, Newton from a = e0 on the KKT system with its certificate
 * that the multiplier lies above lambda_max(A), else FP32 Jacobi + secular);
 * MCG_F64: the solve of the exact FP64 sweep.  In the hard case (b orthogonal
 * to the top eigenspace, a maximum that is not unique) any maximiser may be
 * returned.  n = 0 does nothing; n < 0, a null array (n > 0) or another
 * precision return MCG_BAD_ARG.  Asynchronous on `stream`.
 */
int mcg_local_solve(const double* A, const double* b, double* a_out, int* fallback_out, int n, int precision,
                    cudaStream_t stream);

/*
 * Haar-random gauge transforms (a random Gribov copy U -> G U G^dag(x+mu)
 * with mcg_apply_gauge; Gribov copies: Sec. I and II.B): G(x) in
 * SU(3) for every site x of each of lat->nfields fields (FP64 only; the same
 * matrices in every field).  Site x (lexicographic, x0 fastest) draws
 * Philox4x64-10 (Salmon et al., SC'11) at counters (x, seq, j, 0), j = 0..2,
 * under key (seed, 0x52414E44); u = (w >> 11) 2^-53; Box-Muller on the pairs
 * (1 - u_2i, u_2i+1) gives two complex Gaussian rows, Gram-Schmidt rows 0
 * and 1, row 2 = conj(row0 x row1).  Asynchronous on `stream`.  MCG_BAD_ARG
 * for MCG_F32 fields or a NULL G.
 */
int mcg_random_gauge(void* G, const mcg_lattice* lat, unsigned long long seed, unsigned long long seq,
                     cudaStream_t stream);

/*
 * Simulated annealing of the gauge transform: a Gribov-copy search variant
 * run ahead of mcg_fix (Sec. III.B names annealing as the route to higher maxima
 * taken in SU(2); the paper does not specify it, so this is the library's
 * reading).  For k = 0 .. nsweeps-1: an even then an odd checkerboard
 * half-sweep at temperature T[k]; at each site and for the subgroups (0,1),
 * (0,2), (1,2) in turn, nhit Metropolis hits on the move of mcg_fix
 * (U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dag, Omega(x) <- G Omega(x))
 * with target density exp(F / T), F = sum over the 8 links at x of |tr|^2.
 * Hit h of subgroup s at lexicographic site x in field f of sweep number
 * first_sweep + k draws the four words of Philox4x64-10 at counter
 * (x, first_sweep + k, s * nhit + h, f) under key (seed, 0); u_i = (w_i >> 11)
 * 2^-53; the proposal is a = (sqrt(1 - |v|^2), v), v_i = eps (2 u_i - 1)
 * (i = 0..2), the SU(2) element a0 + i v.sigma in rows/columns of the
 * subgroup; it is accepted when dF >= 0 or u_3 < exp(dF / T).  After the last
 * sweep links and Omega are re-unitarised.  In place on U and G (FP64 fields
 * of lat, fields contiguous; lat->precision must be MCG_F64).
 * T: host, nsweeps temperatures > 0.  nhit in 1..2^20, eps in (0, 0.5].
 * accepted_out: host, nfields, may be NULL: accepted hits per field (out of
 * nsweeps * V * 3 * nhit).  A call with first_sweep = the sweeps done so far
 * continues the same random stream.  Synchronises.
 */
int mcg_anneal(void* U, void* G, const mcg_lattice* lat, const double* T, int nsweeps, long long first_sweep,
               int nhit, double eps, unsigned long long seed, long long* accepted_out, cudaStream_t stream);

/* Z3 center projection (Sec. II.A): m_mu(x) in {-1,0,1} is the sector of
 * phi = arg tr U_mu(x) nearest 2 pi m / 3 (equivalently the closest center
 * element on the group manifold); ties on |phi| = pi/3 go to 0, phi = pi to
 * +1.  The decision is taken in FP64 for both precisions.  Then P-vortices:
 * a plaquette is pierced when (m_mu(x) + m_nu(x+mu) - m_mu(x+nu) - m_nu(x))
 * mod 3 != 0.  Z: device int8 (layout above).  counts: host, 7 x nfields
 * long long: [total, planes 01, 02, 03, 12, 13, 23] per field.  Synchronises. */
int mcg_center_project(const void* U, int8_t* Z, long long* counts, const mcg_lattice* lat,
                       cudaStream_t stream);

/*
 * Center decomposition of a fixed field (Sec. III.A): with Z the center
 * sectors of U (from mcg_center_project, same batch), U_removed <- Z^dag U
 * (the vortex-removed field U' of the paper) and U_center <- Z times the
 * identity (the vortex-only field), in the link layout and precision of U.
 * Either output may be NULL (not both); U_removed may be U itself (in place)
 * but may not overlap it otherwise; U_center may not overlap U or U_removed.
 * conj(Z) multiplies each entry with the products and sums rounded
 * separately (Z = 1 or -1/2 +- i sqrt(3)/2 as literals).  Device pointers;
 * asynchronous on `stream`.
 */
int mcg_vortex_remove(const void* U, const int8_t* Z, void* U_removed, void* U_center, const mcg_lattice* lat,
                      cudaStream_t stream);

/*
 * Planar Wilson loops (Sec. III.A): W(R, T) is the mean over all V
 * translations and the three spatial axes i of
 *   (1/3) Re tr [ S_i^R(x) S_t^T(x + R i) S_i^R(x + T t)^dag S_t^T(x)^dag ],
 * S_mu^L(x) = U_mu(x) U_mu(x+mu) ... U_mu(x+(L-1)mu), t the fourth axis
 * (mu = 3), for 1 <= R <= Rmax (at most the smallest spatial extent) and
 * 1 <= T <= Tmax (at most N_t).  On-axis loops only: the paper's off-axis
 * spatial paths are not built.  Arithmetic in the field's precision, sums in
 * FP64.  W_out: host, nfields x Rmax x Tmax doubles, [f][R-1][T-1].  Uses
 * library scratch of (Tmax + 6) x 9V complex numbers.  Synchronises.
 */
int mcg_wilson_loops(const void* U, const mcg_lattice* lat, int Rmax, int Tmax, double* W_out, cudaStream_t stream);

/*
 * Wilson loops with off-axis spatial sides (Sec. III.A, which uses off-axis
 * paths for non-integer separations without fixing them; this library's
 * reading): for each integer vector r of `vectors` (host, nvec x 3) and
 * 1 <= T <= Tmax (at most N_t), the mean over all translations x and all
 * distinct images r' of r under axis permutations and sign flips of
 *   (1/3) Re tr [ P_r'(x) S_t^T(x + r') P_r'(x + T t)^dag S_t^T(x)^dag ],
 * P_r'(x) the product of links along the lattice path from x to x + r' that
 * steps, at step k of L = |r'0|+|r'1|+|r'2|, along the axis j with the largest
 * deficit k |r'_j| / L - n_j (n_j: steps taken along j; ties to the lowest
 * axis), backward steps contributing U^dag; on-axis r gives mcg_wilson_loops.
 * Each |r_j| must be below the smallest spatial extent, 1 <= L <= 64.
 * W_out: host, nfields x nvec x Tmax doubles.  Uses the same scratch as
 * mcg_wilson_loops.  Synchronises.
 */
int mcg_wilson_loops_offaxis(const void* U, const mcg_lattice* lat, const int* vectors, int nvec, int Tmax,
                             double* W_out, cudaStream_t stream);

/*
 * The preconditioning pipeline of Sec. II.B for every field of the batch:
 * S = smear(U, rho, eps, nsmear); fix S (transform Omega_1 from identity);
 * apply Omega_1 (re-unitarised) to the original U; fix that field (transform
 * Omega_2); center-project and count P-vortices.  nsmear = 0 skips smearing
 * and the first fix (plain MCG).  On return U holds the fixed field and G
 * the total transform Omega_2 Omega_1, so U_out = U_in^G.  smear_precision
 * selects FP64 or FP32 smearing (the smeared field only builds Omega_1).
 * Z (device int8, may be NULL): center sectors of the final field.
 * results: host, nfields entries.  Returns MCG_OK or MCG_NOT_CONVERGED.
 */
int mcg_precondition_fix(void* U, void* G, int8_t* Z, const mcg_lattice* lat, const mcg_params* params,
                         double rho, double eps, int nsmear, int smear_precision, mcg_precond_result* results,
                         cudaStream_t stream);

/*
 * The Sec. II.B experiment over several preconditioning levels of one field,
 * batched: Sec. III scans the number of smearing sweeps (0, 4, ..., 20), each
 * preconditioning conducted independently from the same original field.
 * One smearing chain of U produces the smeared field at every requested level
 * (nsmear: host array, nlevels entries, non-decreasing; 0 = no
 * preconditioning); the smeared fields and the copies of U for the levels
 * without smearing are MCG-fixed as one batch; each smeared level's
 * transform (re-unitarised) is applied to a copy of U; those preconditioned
 * copies are MCG-fixed as a second batch; then center projection, P-vortex
 * counts and plaquettes per level.  Each field's result does not depend on
 * the batch it is fixed in.
 * U: one input field (lat->nfields must be 1), not modified.
 * U_out: nlevels fields (device) receiving the fixed fields; G_out: nlevels
 * transforms (U_out[l] = U^G_out[l]); Z_out (device int8, nlevels fields, may
 * be NULL): center sectors.  results: host, nlevels entries.
 * Returns MCG_OK or MCG_NOT_CONVERGED.  Synchronises.
 */
int mcg_precondition_levels(const void* U, void* U_out, void* G_out, int8_t* Z_out, const mcg_lattice* lat,
                            const mcg_params* params, double rho, double eps, const int* nsmear, int nlevels,
                            int smear_precision, mcg_precond_result* results, cudaStream_t stream);

/*
 * One FP64 half-sweep (exact local maximisation, as mcg_fix's FP64 sweeps) of
 * the sites of `parity` whose t lies in [t_lo, t_hi): the compute step of a
 * lattice split into t-slabs, one per process (domain decomposition; the
 * caller's array is a slab plus ghost layers of the neighbouring slabs'
 * links, which the sites read and update like any other link).  One field,
 * MCG_F64, in place on U and G.  R_out (host, may be NULL): the sum of
 * |tr U|^2 over the 8 links of every updated site, after the update
 * (synchronises); summed over the slabs' odd half-sweeps it is the lattice's
 * R, since every link has exactly one odd end.  Same-parity sites share no
 * link (Sec. II.A checkerboard), so the slabs' half-sweeps together equal the
 * lattice's.
 */
int mcg_halfsweep_slab(void* U, void* G, const mcg_lattice* lat, int parity, int t_lo, int t_hi, double* R_out,
                       cudaStream_t stream);

/*
 * The halo face of a t-slab (domain decomposition of the Sec. II.A
 * relaxation): the forward t-links U_t(x) (mu = 3, all nine entries) of the
 * sites of one t-layer and one checkerboard parity, copied between a field
 * and a contiguous buffer on the device.  A half-sweep of parity P reads the
 * t-link of a first-layer site's backward neighbour, which lies on the last
 * layer of the slab below and has parity 1 - P: that face is the one
 * message each way per half-sweep.
 * U: one field (lat->nfields must be 1), MCG_F64 or MCG_F32, device.
 * t: the layer, 0 <= t < N_t; parity: 0 or 1, the parity of the sites in
 * U's own checkerboard.  buf: device, 9 * (N_x N_y N_z / 2) elements of U's
 * type (complex, 16 or 8 bytes), entry-major: buf[e * n + i] is entry
 * e = 3*row + col of the i-th site of the face, sites in (x, y, z)
 * lexicographic order (x fastest) -- the same order on both sides of a slab
 * boundary, so a face read from layer L of one slab is written unchanged into
 * layer 0 of the next.  to_field: 0 copies U -> buf, 1 copies buf -> U (only
 * the face's t-links change).  buf must not overlap U.  Asynchronous on
 * `stream` (one pitched device-to-device copy).
 * Returns MCG_OK, MCG_BAD_DIMS, MCG_BAD_ARG or MCG_CUDA_ERROR.
 */
int mcg_slab_face(void* U, void* buf, const mcg_lattice* lat, int t, int parity, int to_field, cudaStream_t stream);

/*
 * Index checks (not in the paper: a debugging aid).  In a library built with
 * -DMCG_CHECK (paper_0807_0264_gb300.build.build(check=True)) the kernels'
 * layout helpers test every index against its array; an index out of range
 * is counted and replaced by a valid one, so the access stays inside the
 * array and no kernel traps.  Returns the number of such indices met since
 * the last reset (synchronises the device; reset != 0 zeroes the counters),
 * or -1 in a regular build (no device call).
 */
long long mcg_bounds_violations(int reset);

/*
 * MCG relaxation (as mcg_fix) of a batch of fields of any sizes, all of one
 * precision: each field's half-sweeps run as their own chain of launches
 * (the chains concurrent inside one graph per chunk of sweeps); a field stops
 * (its blocks exit at entry) once it has converged.  fields: host array of
 * nfields entries.  R_out / sweeps_out: host, nfields entries (may be NULL).
 * Returns MCG_OK when every field converged, else MCG_NOT_CONVERGED.
 */
int mcg_fix_batch(const mcg_field* fields, int nfields, int precision, const mcg_params* params, double* R_out,
                  int* sweeps_out, cudaStream_t stream);

/*
 * Gribov-copy search (Sec. I: MCG fixing is plagued by Gribov copies, and
 * higher maxima of the functional change the vortex content): for every copy,
 * U (device) holds its configuration's links and G (device) a random initial
 * transform Omega0; the call applies Omega0 (U <- U^Omega0), fixes all copies
 * of all configurations as one batch (G then holds each copy's total
 * transform, U = U_config^G), and picks per configuration the copy with the
 * largest V_U (ties keep the lower copy index).  config_of_copy: host,
 * ncopies entries in [0, nconfigs).  R_out / sweeps_out: host, per copy (may
 * be NULL); best_copy / best_V: host, per configuration (may be NULL).
 * Returns MCG_OK or MCG_NOT_CONVERGED.  Synchronises.
 */
int mcg_gribov_search(const mcg_field* copies, int ncopies, const int* config_of_copy, int nconfigs, int precision,
                      const mcg_params* params, double* R_out, int* sweeps_out, int* best_copy, double* best_V,
                      cudaStream_t stream);

/* ---- differentiation (not in the paper: the training pattern that
 * differentiates the method) ------------------------------------------------
 * Matrix-gradient convention: for a real loss L and a link U,
 * G = dL/dRe U + i dL/dIm U (dL = Re tr(G^dag dU)); G arrays are FP64 in the
 * link layout, i.e. the (re, im) pairs a real-view autograd gradient holds.
 * The derivative along U -> exp(i eta T_a) U is Re tr(G^dag i T_a U). */

/* Reverse-mode derivative of one smearing step U' = exp(iQ(U)) U (the step of
 * mcg_smear, Sec. II.B): Gin = gradient w.r.t. U given Gout w.r.t. U'.
 * Chain rule per link: Gin += exp(iQ)^dag Gout; the adjoint of exp's Frechet
 * derivative B = L(iQ, U Gout^dag); its traceless anti-Hermitian part K; then
 * Gin += K C on the link and rho U^dag K scattered over every factor of every
 * staple (atomic FP64 adds: summation order, hence the last bits, vary).
 * U: the step's input field (FP64); Gout, Gin: FP64, link layout, distinct. */
int mcg_smear_backward_step(const void* U, const double* Gout, double* Gin, const mcg_lattice* lat, double rho,
                            double eps, cudaStream_t stream);

/* Matrix gradient of R = sum |tr U|^2 (Sec. II.A): G = 2 tr(U) 1 per link. */
int mcg_functional_matrix_grad(const void* U, double* G, const mcg_lattice* lat, cudaStream_t stream);

/* Lie-algebra gradient of R with respect to the gauge transform:
 * grad[f][i][a] = dR/d eps for Omega(x_i) -> exp(i eps lambda_a/2) Omega(x_i),
 * i the lexicographic site index, a = 0..7 (Gell-Mann order).  FP64, device. */
int mcg_grad_R(const void* U, double* grad, const mcg_lattice* lat, cudaStream_t stream);

/* Gradient-ascent step on the gauge transform: W(x) = exp(i alpha sum_a
 * grad_a(x) lambda_a/2), Omega(x) <- W(x) Omega(x), U_mu(x) <- W(x) U_mu(x)
 * W(x+mu)^dag for all sites at once (uses library scratch for W). */
int mcg_ascent_step(void* U, void* G, const double* grad, double alpha, const mcg_lattice* lat, cudaStream_t stream);

/* ---- measurement ---------------------------------------------------------- */

/* Mean duration of one launch of the half-sweep kernel (parity 0: even sites;
 * parity 1: odd sites with the fused R reduction) on one field, over nreps
 * launches each bracketed by CUDA events on `stream`; with flush_l2 != 0 a
 * 256 MB buffer is overwritten between launches, outside the timed interval,
 * so every launch reads its links from HBM.  FP64: the sweeps are applied to
 * U and G.  FP32: the FP32 kernel works on the library's compact storage
 * (rows 0 and 1 of each matrix, row 2 implied by unitarity); U and G are
 * converted to it once, before the timed launches, and left unchanged.
 * ms_out: host float.  Synchronises.  (Instrumentation; not part of the
 * paper's method.) */
int mcg_time_halfsweep(void* U, void* G, const mcg_lattice* lat, int parity, int nreps, int flush_l2, float* ms_out,
                       cudaStream_t stream);

/*
 * Mean plaquette per field, like mcg_plaquette, for callers that cannot let
 * the library allocate device memory (the paper has no counterpart: this is
 * an interface variant).  Its only scratch, the per-block partial sums, is a
 * fixed 512 KiB array compiled into the library (65 536 doubles), so a call
 * needs nfields * ceil(V / 256) <= 65 536; larger requests return
 * MCG_BAD_ARG without touching the GPU.  out: DEVICE pointer to nfields
 * doubles, written asynchronously on `stream` (no synchronisation, no host
 * transfer).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address stays cached for the process;
 * after a cudaDeviceReset call mcg_release() (which drops the cache) before
 * the next call.  All calls share the one array and it keeps
 * the previous call's partial sums: calls whose kernels overlap on the GPU
 * (other streams, other host threads) race and must be ordered by the caller.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 */
int mcg_plaquette_static(const void* U, double* out, const mcg_lattice* lat, cudaStream_t stream);

/* Threads per block of the half-sweep kernel for one precision, one thread
 * per site: FP64 64 or 128, FP32 64, 128 or 256; 128 by default.  A process-wide tuning setting (not part of the paper's
 * method): Python's autotune_sweep_block() times the choices with
 * mcg_time_halfsweep and keeps the fastest.  Returns MCG_BAD_ARG otherwise. */
int mcg_set_sweep_block(int precision, int threads);
int mcg_get_sweep_block(int precision);

/* Running total of CUDA kernels this library has enqueued in this process
 * (kernels inside a CUDA graph count once per graph launch). */
long long mcg_kernel_launches(void);

/* Sweep-phase accounting since the last reset (instrumentation; not part of
 * the paper's method): ms_out[p] = GPU milliseconds of the relaxation's sweep
 * graphs (half-sweeps, end-of-sweep reductions, FP64 re-unitarisation), timed
 * with CUDA events on the calling stream, and site_updates_out[p] = sites x
 * half-sweeps they performed (a full sweep of a field is V site-updates),
 * for p = 0: FP64 sweeps, p = 1: FP32 sweeps.  ms_out: host, 2 doubles;
 * site_updates_out: host, 2 long long.  reset != 0 zeroes the counters. */
int mcg_phase_stats(double* ms_out, long long* site_updates_out, int reset);

/* Arithmetic throughput of the current device (instrumentation, the
 * denominators of ALU-bound kernels): tflops_out[0] = FP64 FMA, [1] = FP32
 * FMA, [2] = packed FP32 FMA (two FMAs on a register pair), in TFLOP/s at
 * 2 flop per FMA, each from ~20 ms of independent FMA chains in every thread
 * of 8 blocks of 256 per SM, timed with CUDA events.  tflops_out: host, 3
 * doubles.  Synchronises. */
int mcg_probe_peaks(double* tflops_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MCG_H */
