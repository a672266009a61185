// Host-side internals shared by the libmcg translation units (not part of the
// public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <functional>

#include <string>
#include <vector>

#include "mcg_common.cuh"

namespace mcg {

// ---- error reporting ------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define MCG_CK(call)                                          \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::mcg::cuda_fail(e_, #call); \
    } while (0)

// ---- argument checks ----------------------------------------------------------
// Validates a lattice descriptor (even extents in [2, 32768], at most 2^30
// sites per parity, 1..2^20 fields, a known precision) and fills g.
int check_lattice(const mcg_lattice* lat, Geom* g);

// Drops the cached device addresses of the allocation-free entry point's
// static array (mcg_release calls it).
void static_release();

// ---- launch accounting ------------------------------------------------------
// Every kernel the library enqueues is counted (graph launches count their
// kernel nodes); mcg_kernel_launches() reports the running total.
void note_launches(long long n);
// Sweep-phase accounting: GPU milliseconds of the sweep graphs and the
// site-updates they performed, per precision (mcg_phase_stats reports them).
void note_phase(int prec, double ms, long long site_updates);

// ---- scratch ----------------------------------------------------------------
// Named, grow-only device and pinned-host buffers cached per device; freed by
// mcg_release().
void* scratch_device(const char* name, size_t bytes, int* rc);
void* scratch_host(const char* name, size_t bytes, int* rc);
cudaStream_t capture_stream(int* rc);
// n branch streams (and an event per stream, plus a fork event) for the
// per-field chains of a captured sweep graph, cached per device.
int branch_streams(int n, cudaStream_t* streams, cudaEvent_t* events, cudaEvent_t* fork, int* rc);
// index-check counters of the kernel units (0 unless built with MCG_CHECK)
unsigned long long bound_hits_field(bool reset);
unsigned long long bound_hits_observables(bool reset);
unsigned long long bound_hits_smear(bool reset);
unsigned long long bound_hits_sweep(bool reset);
unsigned long long bound_hits_sweep_f32(bool reset);
unsigned long long bound_hits_sweep_df(bool reset);
void release_all();

// ---- batched sweep machinery -------------------------------------------------
struct FieldDesc {
    void* U;      // links: FP64 full layout, or FP32 compact (rows 0 and 1)
    void* G;      // gauge transform, same storage as the links
    Geom geo;
    int blk0;     // first block of this field in the flattened grid
    int nblk;     // blocks of this field
    double norm;  // 1 / (9 * 4V)
    void* Ulo = nullptr;  // double-float storage: the lo parts of U and G (U, G
    void* Glo = nullptr;  // then hold the hi parts), compact layout
    int t_lo = 0;         // FP64 half-sweep: only sites with t_lo <= t < t_hi
    int t_hi = 1 << 30;   // (a t-slab of a decomposed lattice)
    double omega = 1.0;   // FP32 (compact) sweeps: this field's over-relaxation
};

// Tag of the double-float sweep phase in run_fix_phase<T> (T = float: compact
// FP32, double: FP64 full layout, DoubleFloat: compact hi + lo FP32 pairs).
struct DoubleFloat {};

constexpr int kRing = 32;  // R history kept per field for windowed stop tests

struct FieldState {
    double R_prev;  // R after the previous sweep (or at phase start)
    double R_last;  // R after the last sweep
    int sweep;      // sweeps completed (across phases)
    int done;       // 0 running, 1 converged, 2 sweep cap of the phase reached
    int reunit_pending;
    int max_sweeps;   // absolute sweep cap of the current phase
    int fallbacks;    // local solves that needed the FP64 fallback path
    int phase_start;  // sweep count when the current phase began
    double ring[kRing];  // R after sweep k stored at k % kRing
};

struct SweepBatch {
    const FieldDesc* desc;
    int nf;
    int total_blocks;
    FieldState* state;
    double* partial;  // one per warp: ppb per block
    int ppb;          // partials per block (threads per block / 32)
    double* R_hist;   // nf x hist_len (may be null)
    int hist_len;
    double tol;
    int window;  // stop when the dV_U averaged over `window` sweeps < tol
    int reunit_every;
    double omega;  // over-relaxation parameter (1: plain relaxation)
    int solve32;   // FP64 sweeps: local problem built and solved in FP32
};

// Haar-random SU(3) transforms (FP64 gauge layout, the same in each of the
// nfields; Philox4x64-10 with key (seed, 0x52414E44), counter (x, seq, j, 0)),
// and G <- W G per site (FP64; W one field).
int launch_random_gauge(void* G, const Geom& g, int nfields, unsigned long long seed, unsigned long long seq,
                        cudaStream_t st);
int launch_gauge_left_mul(void* G, const void* W, const Geom& g, int nfields, cudaStream_t st);

// Restarts of the FP32 (compact) phase: a field that has run `after` sweeps
// since its last (re)start without stopping gets its working copies reset by
// reset(f, k, stream) (k its restart count, from 1; enqueued on the phase's
// stream) and continues with the
// over-relaxation omega_k of its k-th restart, k = 1, 2, ...: omega - d,
// omega + d, omega - 2d, omega + 2d, ... (d = domega); no restart once
// omega_k leaves (0, 2).  Its sweeps keep counting toward the phase's cap.
// count (nf entries, may be null): restarts per field.
// A field also restarts when it creeps: over the last `creep` sweeps (0:
// off) the mean dV_U per sweep of every check_every chunk stayed within
// [creep_lo, creep_hi] and the mean of the last quarter of those chunks is
// more than half the mean of the first quarter (no decay); see creeping().
struct PhaseRestart {
    int after = 0;
    double domega = 0.0;
    std::function<int(int, int, cudaStream_t)> reset;
    int* count = nullptr;
    int creep = 0;
    double creep_lo = 0.0, creep_hi = 0.0;
};

// The creep test on the per-chunk dV_U of the last m chunks, oldest first.
inline bool creeping(const double* dv, int m, double lo, double hi) {
    if (m < 4) return false;
    const int q = m / 4;
    double first = 0.0, last = 0.0;
    for (int i = 0; i < m; ++i) {
        if (!(dv[i] >= lo && dv[i] <= hi)) return false;
        if (i < q) first += dv[i];
        if (i >= m - q) last += dv[i];
    }
    return last > 0.5 * first;
}

// Over-relaxation of a field's k-th restart (k = 0: the phase's own), or a
// value outside (0, 2) when there is none.
inline double restart_omega(double omega, double domega, int k) {
    const int m = (k + 1) / 2;
    return omega + (k % 2 ? -1.0 : 1.0) * m * domega;
}

// Run MCG relaxation on a batch (all fields same precision T) until every
// field is done: converged (dV_U < tol) or at abs_cap sweeps counted from the
// start of the history.  `fresh`: start a new history (sweep = 0); otherwise
// continue the sweep count in `state` (a new phase).  restart (T = float
// only, may be null): see PhaseRestart.  Returns 0 or an error.
template <typename T>
int run_fix_phase(const std::vector<FieldDesc>& fields, FieldState* d_state, FieldState* h_state, double* d_hist,
                  int hist_len, double tol, int window, double omega, int reunit_every, int abs_cap,
                  int check_every, bool fresh, cudaStream_t stream, bool solve32 = false,
                  const PhaseRestart* restart = nullptr);

// Time `nreps` launches of one half-sweep kernel (parity 1 includes the fused
// R reduction) on a single field, each bracketed by CUDA events on `stream`;
// with flush_l2 a 256 MB buffer is overwritten between launches (outside the
// timed interval).  Returns the mean per-launch milliseconds in *ms.
template <typename T>
int time_halfsweep(void* U, void* G, const Geom& g, int parity, int nreps, int flush_l2, float* ms,
                   cudaStream_t stream);

// n local problems (A16: n row-major 4x4 matrices, upper triangle read; b4:
// n 4-vectors) solved on the device by the FP32 sweeps' solve (prec MCG_F32)
// or the exact FP64 sweep's (MCG_F64): a4 the maximisers, fb (may be null) 1
// where the solve left the Newton path.
int launch_local_solve(const double* A16, const double* b4, double* a4, int* fb, int n, int prec, cudaStream_t st);

// One FP64 half-sweep (exact local solve) of the sites of `parity` with
// t_lo <= t < t_hi on one field; want_R: the odd-parity R partial of those
// sites' 8 links to *R_host (synchronises).
int run_halfsweep_slab(void* U, void* G, const Geom& g, int parity, int t_lo, int t_hi, bool want_R, double* R_host,
                       cudaStream_t stream);

// Simulated annealing (FP64 fields of one lattice, fields contiguous): for
// k < nsweeps an even then an odd Metropolis half-sweep at temperature T[k]
// (host array) with sweep number first_sweep + k in the random counter; then
// links and Omega are re-unitarised.  accepted_host (nfields, may be null):
// accepted hits per field.  Synchronises.
int run_anneal(void* U, void* G, const Geom& g, int nfields, const double* T, int nsweeps, long long first_sweep,
               int nhit, double eps, unsigned long long seed, long long* accepted_host, cudaStream_t st);

// The double-float half-sweep (mcg_sweep_df.cu): threads (= sites) per block,
// shared-memory set-up, launches of the half-sweep and of the R reduction,
// FP64 full layout -> double-float compact links, identity transform.
int df_threads();
int prepare_halfsweep_df();
void launch_halfsweep_df(bool acc, const SweepBatch& bt, int parity, int nblocks, cudaStream_t st);
void launch_functional_df(const SweepBatch& bt, int nblocks, cudaStream_t st);
int launch_to_df(const double* src, void* hi, void* lo, const Geom& g, int nmat, int nfields, cudaStream_t st);
int launch_identity_df(void* hi, void* lo, const Geom& g, int nfields, cudaStream_t st);

// The compact FP32 half-sweep (mcg_sweep_f32.cu): raise its shared-memory
// limit for nt threads per block (64, 128, 256) on the current device, and
// launch one half-sweep of the batch (acc: with the fused R partials).
int prepare_halfsweep_c12(int nt);
void launch_halfsweep_c12(int nt, bool acc, const SweepBatch& bt, int parity, int nblocks, cudaStream_t st);

// threads per block of the half-sweep kernel for a precision, and the sites
// each block covers (one thread per site in both precisions)
int sweep_block(int prec);
void set_sweep_block(int prec, int nt);
int sweep_sites_per_block(int prec);

// ---- input validation (mcg_field.cu) -----------------------------------------
// Tolerances of the SU(3) check on caller-supplied fields: max |M M^dag - 1|
// and |det M - 1|.  Far above rounding (FP64 fields ~1e-15, FP32 ~1e-7), far
// below any real defect (a link scaled by 1.01 is off by 2e-2).
constexpr float kSU3TolF64 = 1e-6f;
constexpr float kSU3TolF32 = 1e-4f;
// Checks every matrix of nfields fields (nslots = 8 for links, 2 for gauge
// transforms); returns 0, or MCG_BAD_INPUT with a message naming `what` and
// the first failing matrix.  finite_only: only finiteness is required.
// Synchronises the stream.
int validate_su3(const void* M, int prec, const Geom& g, int nslots, int nfields, const char* what,
                 cudaStream_t st, bool finite_only = false);

// Arithmetic throughput probes: tflops[0..2] = FP64 FMA, FP32 FMA, packed FP32
// FMA (TFLOP/s, 2 flop per FMA lane), measured on the current device.
int probe_peaks(double* tflops, cudaStream_t st);

// ---- field kernels (mcg_field.cu) -------------------------------------------
int launch_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t n, cudaStream_t st);
int launch_identity_gauge(void* G, int prec, const Geom& g, int nfields, cudaStream_t st);
int launch_apply_gauge(void* U, const void* G, int prec, const Geom& g, int nfields, cudaStream_t st);
int launch_reunitarise(void* M, int which, int prec, const Geom& g, int nfields, cudaStream_t st);
int compute_plaquette(const void* U, int prec, const Geom& g, int nfields, double* out_host, cudaStream_t st);
int compute_functional(const void* U, int prec, const Geom& g, int nfields, double* out_host, cudaStream_t st);
int compute_center(const void* U, int prec, int8_t* Z, const Geom& g, int nfields, long long* counts_host,
                   cudaStream_t st);
// FP32 transform W of this call (compact form) -> FP64: W64 = reunit(W);
// U64 <- W64 U64 W64(x+mu)^dag; G64 <- reunit(W64 G64).  W32lo (may be null):
// lo parts of a double-float W (W = hi + lo).
int launch_handoff(const void* W32, const void* W32lo, double* U64, double* G64, const Geom& g, int nfields,
                   cudaStream_t st);
// compact FP32 working storage (rows 0 and 1 of each matrix) of the FP32
// sweep phase: from / to the full layout; nmat = 4 for links, 1 for a gauge
// transform
int launch_to_c12(const void* src, int src_prec, void* dst, const Geom& g, int nmat, int nfields, cudaStream_t st);
int launch_from_c12(const void* src, void* dst, const Geom& g, int nmat, int nfields, cudaStream_t st);
int launch_identity_c12(void* W, const Geom& g, int nfields, cudaStream_t st);

// ---- center decomposition and Wilson loops (mcg_observables.cu) --------------
int launch_vortex_remove(const void* U, const int8_t* Z, void* Ur, void* Zl, int prec, const Geom& g, int nfields,
                         cudaStream_t st);
int compute_wilson_loops(const void* U, int prec, const Geom& g, int nfields, int Rmax, int Tmax, double* W_host,
                         cudaStream_t st);
int compute_wilson_loops_offaxis(const void* U, int prec, const Geom& g, int nfields, const int* vecs, int nvec,
                                 int Tmax, double* W_host, cudaStream_t st);

// ---- smearing (mcg_smear.cu) ------------------------------------------------
int run_smear(const void* Uin, void* Uout, int prec, const Geom& g, int nfields, double rho, double eps, int n,
              cudaStream_t st);

// ---- differentiation (mcg_smear.cu) -----------------------------------------
int run_smear_step_backward(const void* U, const double* Gout, double* Gin, const Geom& g, int nfields, double rho,
                            double eps, cudaStream_t st);
int run_functional_matrix_grad(const void* U, int prec, double* G, const Geom& g, int nfields, cudaStream_t st);
int run_grad_R(const void* U, int prec, double* grad, const Geom& g, int nfields, cudaStream_t st);
int run_ascent_step(void* U, void* G, const double* grad, double alpha, int prec, const Geom& g, int nfields,
                    cudaStream_t st);

}  // namespace mcg
