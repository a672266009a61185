// The extern "C" boundary of libmcg (declared in include/mcg.h): argument
// validation, error reporting, scratch management and the host-side
// orchestration of the MCG relaxation and the preconditioning pipeline.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mcg.h"
#include "mcg_common.cuh"
#include "mcg_internal.h"

namespace mcg {

int launch_pack(const double* canon, void* soa, int prec, const Geom& g, int nfields, int what, int unpack,
                cudaStream_t st);
int launch_unpack_center(const int8_t* Z, int8_t* canon, const Geom& g, int nfields, cudaStream_t st);

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    set_error(buf);
    return MCG_CUDA_ERROR;
}

// ---------------------------------------------------------------------------
// NVTX ranges (header-only NVTX 3: no cost unless a profiler is attached)
// ---------------------------------------------------------------------------
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// launch accounting
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_phase_mu;
static double g_phase_ms[2] = {0.0, 0.0};
static long long g_phase_su[2] = {0, 0};
void note_phase(int prec, double ms, long long site_updates) {
    std::lock_guard<std::mutex> lk(g_phase_mu);
    const int i = prec == MCG_F64 ? 0 : 1;
    g_phase_ms[i] += ms;
    g_phase_su[i] += site_updates;
}

// ---------------------------------------------------------------------------
// scratch: grow-only named buffers per device
// ---------------------------------------------------------------------------
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};
struct DeviceScratch {
    std::map<std::string, Buf> dev, host;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;  // branch streams of captured per-field chains
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t fork_ev = nullptr;
};
static std::mutex g_mu;
static std::map<int, DeviceScratch> g_scratch;

static DeviceScratch& cur(int* rc) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) *rc = cuda_fail(e, "cudaGetDevice");
    return g_scratch[d];
}

void* scratch_device(const char* name, size_t bytes, int* rc) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch& ds = cur(rc);
    if (*rc) return nullptr;
    Buf& b = ds.dev[name];
    if (b.bytes < bytes) {
        if (b.p) {
            cudaDeviceSynchronize();
            cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) {
            *rc = cuda_fail(e, "cudaMalloc(scratch)");
            return nullptr;
        }
        b.bytes = std::max<size_t>(bytes, 256);
    }
    return b.p;
}

void* scratch_host(const char* name, size_t bytes, int* rc) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch& ds = cur(rc);
    if (*rc) return nullptr;
    Buf& b = ds.host[name];
    if (b.bytes < bytes) {
        if (b.p) {
            cudaDeviceSynchronize();
            cudaFreeHost(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMallocHost(&b.p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) {
            *rc = cuda_fail(e, "cudaMallocHost(scratch)");
            return nullptr;
        }
        b.bytes = std::max<size_t>(bytes, 256);
    }
    return b.p;
}

cudaStream_t capture_stream(int* rc) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch& ds = cur(rc);
    if (*rc) return nullptr;
    if (!ds.cap) {
        cudaError_t e = cudaStreamCreateWithFlags(&ds.cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            *rc = cuda_fail(e, "cudaStreamCreate");
            return nullptr;
        }
    }
    return ds.cap;
}

int branch_streams(int n, cudaStream_t* streams, cudaEvent_t* events, cudaEvent_t* fork, int* rc_out) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = 0;
    DeviceScratch& ds = cur(&rc);
    if (rc) return *rc_out = rc;
    cudaError_t e = cudaSuccess;
    if (!ds.fork_ev) e = cudaEventCreateWithFlags(&ds.fork_ev, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)ds.side.size() < n) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (s) ds.side.push_back(s);
        if (ev) ds.side_ev.push_back(ev);
    }
    if (e != cudaSuccess) return *rc_out = cuda_fail(e, "branch streams");
    for (int i = 0; i < n; ++i) {
        streams[i] = ds.side[i];
        events[i] = ds.side_ev[i];
    }
    *fork = ds.fork_ev;
    return *rc_out = 0;
}

void release_all() {
    static_release();
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    for (auto& kv : g_scratch) {
        cudaSetDevice(kv.first);
        cudaDeviceSynchronize();
        for (auto& b : kv.second.dev)
            if (b.second.p) cudaFree(b.second.p);
        for (auto& b : kv.second.host)
            if (b.second.p) cudaFreeHost(b.second.p);
        if (kv.second.cap) cudaStreamDestroy(kv.second.cap);
        for (auto s : kv.second.side) cudaStreamDestroy(s);
        for (auto ev : kv.second.side_ev) cudaEventDestroy(ev);
        if (kv.second.fork_ev) cudaEventDestroy(kv.second.fork_ev);
    }
    g_scratch.clear();
    cudaSetDevice(dev);
}

// ---------------------------------------------------------------------------
// validation helpers
// ---------------------------------------------------------------------------
// Extents are bounded before they are multiplied (no overflow for any int
// input): each in [2, 32768] and even, V / 2 <= 2^30, 1 <= nfields <= 2^20.
int check_lattice(const mcg_lattice* lat, Geom* g) {
    if (!lat) return fail(MCG_BAD_ARG, "lattice descriptor is NULL");
    for (int d = 0; d < 4; ++d)
        if (lat->dims[d] < 2 || (lat->dims[d] & 1))
            return fail(MCG_BAD_DIMS, "every lattice extent must be even and >= 2");
    for (int d = 0; d < 4; ++d)
        if (lat->dims[d] > (1 << 15)) return fail(MCG_BAD_DIMS, "lattice extent above 32768");
    if (lat->nfields < 1 || lat->nfields > (1 << 20)) return fail(MCG_BAD_DIMS, "nfields must be in [1, 2^20]");
    if (lat->precision != MCG_F64 && lat->precision != MCG_F32)
        return fail(MCG_BAD_ARG, "precision must be MCG_F64 or MCG_F32");
    const long long V = (long long)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
    if (V / 2 > (1LL << 30)) return fail(MCG_BAD_DIMS, "lattice too large");
    for (int d = 0; d < 4; ++d) g->n[d] = lat->dims[d];
    g->vh = (int)(V / 2);
    return 0;
}

static int check_lat(const mcg_lattice* lat, Geom* g) { return check_lattice(lat, g); }

static size_t elem_bytes(int prec) { return prec == MCG_F64 ? 16 : 8; }

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

static int check_params(const mcg_params* p) {
    if (!p) return fail(MCG_BAD_ARG, "params is NULL");
    if (p->fp64_df != 0 && p->fp64_df != 1) return fail(MCG_BAD_ARG, "fp64_df must be 0 or 1");
    if (p->max_sweeps < 0) return fail(MCG_BAD_ARG, "max_sweeps must be >= 0");
    if (p->check_every < 1) return fail(MCG_BAD_ARG, "check_every must be >= 1");
    if (p->reunit_every < 0 || p->fp32_sweeps < 0) return fail(MCG_BAD_ARG, "negative schedule parameter");
    if (p->fp32_sweeps > 0 && !(p->fp32_overrelax > 0.0 && p->fp32_overrelax < 2.0))
        return fail(MCG_BAD_ARG, "fp32_overrelax must be in (0, 2)");
    if (p->fp64_solve32 != 0 && p->fp64_solve32 != 1) return fail(MCG_BAD_ARG, "fp64_solve32 must be 0 or 1");
    if (p->fp32_sweeps > 0 && (p->fp32_window < 1 || p->fp32_window > 31))
        return fail(MCG_BAD_ARG, "fp32_window must be in 1..31");
    if (!(p->tol == p->tol)) return fail(MCG_BAD_ARG, "tol is NaN");
    if (p->fp32_restart < 0 || !(p->fp32_restart_domega >= 0.0 && p->fp32_restart_domega < 2.0))
        return fail(MCG_BAD_ARG, "fp32_restart must be >= 0 and fp32_restart_domega in [0, 2)");
    if (p->fp32_restart_random != 0 && p->fp32_restart_random != 1)
        return fail(MCG_BAD_ARG, "fp32_restart_random must be 0 or 1");
    if (p->fp32_restart_creep < 0) return fail(MCG_BAD_ARG, "fp32_restart_creep must be >= 0");
    if (p->fp32_plain_finish != 0 && p->fp32_plain_finish != 1)
        return fail(MCG_BAD_ARG, "fp32_plain_finish must be 0 or 1");
    return 0;
}

// ---------------------------------------------------------------------------
// MCG fix orchestration
// ---------------------------------------------------------------------------
// One field of a (possibly heterogeneous) batch.
struct FieldSpec {
    void* U;
    void* G;
    Geom g;
};

// MCG relaxation of a batch of fields (all of one precision, any sizes), one
// launch per half-sweep for the whole batch.
static int fix_fields(const std::vector<FieldSpec>& fs, int prec, const mcg_params* prm, double* R_out,
                      int* sweeps_out, int* sweeps32_out, double* R_hist, cudaStream_t st, int* converged_out = nullptr,
                      int* restarts_out = nullptr) {
    const int nf = (int)fs.size();
    int rc = 0;
    FieldState* d_state = (FieldState*)scratch_device("fix.state", sizeof(FieldState) * nf, &rc);
    if (rc) return rc;
    FieldState* h_state = (FieldState*)scratch_host("fix.state", sizeof(FieldState) * nf, &rc);
    if (rc) return rc;
    const int hist_len = prm->max_sweeps + 1;
    double* d_hist = nullptr;
    if (R_hist) {
        d_hist = (double*)scratch_device("fix.hist", sizeof(double) * hist_len * (size_t)nf, &rc);
        if (rc) return rc;
        MCG_CK(cudaMemsetAsync(d_hist, 0, sizeof(double) * hist_len * (size_t)nf, st));
    }
    std::vector<int> s32(nf, 0);
    bool fresh = true;

    // FP32 sweeps run on compact working copies (rows 0 and 1 of each matrix)
    auto compact_copies = [&](std::vector<FieldDesc>& fds, int* rcp) {
        size_t lo_tot = 0, go_tot = 0;
        for (const auto& f : fs) {
            lo_tot += c12_link_chunks(f.g);
            go_tot += c12_gauge_chunks(f.g);
        }
        char* U12 = (char*)scratch_device("fix.U12", 16 * lo_tot, rcp);
        if (*rcp) return;
        char* W12 = (char*)scratch_device("fix.W12", 16 * go_tot, rcp);
        if (*rcp) return;
        fds.resize(nf);
        size_t lo = 0, go = 0;
        for (int f = 0; f < nf; ++f) {
            const Geom& g = fs[f].g;
            fds[f].U = U12 + 16 * lo;
            fds[f].G = W12 + 16 * go;
            fds[f].geo = g;
            fds[f].norm = 1.0 / (9.0 * 8.0 * g.vh);
            lo += c12_link_chunks(g);
            go += c12_gauge_chunks(g);
        }
    };

    if (prec == MCG_F64 && prm->fp32_sweeps > 0) {
        NvtxRange nvtx_phase_("fix: FP32 phase");
        // FP32 phase on compact copies of the links and on the transform W of
        // this call (starting from the identity)
        std::vector<FieldDesc> fds;
        compact_copies(fds, &rc);
        if (rc) return rc;
        for (int f = 0; f < nf; ++f) {
            if ((rc = launch_to_c12(fs[f].U, MCG_F64, fds[f].U, fs[f].g, 4, 1, st))) return rc;
            if ((rc = launch_identity_c12(fds[f].G, fs[f].g, 1, st))) return rc;
        }
        const int cap = std::min(prm->fp32_sweeps, prm->max_sweeps);
        // restarts from this call's input: the FP64 links are untouched until
        // the hand-off
        std::vector<int> nrs(nf, 0);
        PhaseRestart rs;
        rs.after = prm->fp32_restart;
        rs.domega = prm->fp32_restart_domega;
        rs.count = nrs.data();
        void* W0 = nullptr;
        rs.creep = prm->fp32_restart_creep;
        rs.creep_lo = 2.0 * prm->fp32_tol;
        rs.creep_hi = 20.0 * prm->fp32_tol;
        const bool any_restart = prm->fp32_restart > 0 || prm->fp32_restart_creep > 0;
        if (any_restart && prm->fp32_restart_random) {
            size_t ge_max = 0;
            for (const auto& f : fs) ge_max = std::max(ge_max, gauge_elems(f.g));
            W0 = scratch_device("fix.restart.W0", 16 * ge_max, &rc);
            if (rc) return rc;
        }
        rs.reset = [&](int f, int k, cudaStream_t s) -> int {
            int r = 0;
            if (W0) {
                // a random gauge copy of the field: W0 applied to the FP64
                // links, the call's transform left-multiplied by it
                r = launch_random_gauge(W0, fs[f].g, 1, MCG_RESTART_SEED, (unsigned long long)k, s);
                if (!r) r = launch_apply_gauge(fs[f].U, W0, MCG_F64, fs[f].g, 1, s);
                if (!r) r = launch_gauge_left_mul(fs[f].G, W0, fs[f].g, 1, s);
            }
            if (!r) r = launch_to_c12(fs[f].U, MCG_F64, fds[f].U, fs[f].g, 4, 1, s);
            if (!r) r = launch_identity_c12(fds[f].G, fs[f].g, 1, s);
            return r;
        };
        rc = run_fix_phase<float>(fds, d_state, h_state, d_hist, hist_len, prm->fp32_tol, prm->fp32_window,
                                  prm->fp32_overrelax, 0, cap, prm->check_every, true, st, false,
                                  any_restart ? &rs : nullptr);
        if (rc) return rc;
        if (restarts_out)
            for (int f = 0; f < nf; ++f) restarts_out[f] = nrs[f];
        if (prm->fp32_plain_finish && prm->fp32_overrelax != 1.0) {
            // plain FP32 sweeps from where the over-relaxed ones stopped
            rc = run_fix_phase<float>(fds, d_state, h_state, d_hist, hist_len, prm->fp32_tol, prm->fp32_window, 1.0,
                                      0, cap, prm->check_every, false, st);
            if (rc) return rc;
        }
        for (int f = 0; f < nf; ++f) s32[f] = h_state[f].sweep;
        // hand-off: FP64 re-unitarised transform applied to the FP64 links
        for (int f = 0; f < nf; ++f)
            if ((rc = launch_handoff(fds[f].G, nullptr, (double*)fs[f].U, (double*)fs[f].G, fs[f].g, 1, st)))
                return rc;
        fresh = false;
    }
    if (prec == MCG_F64 && prm->fp64_df) {
        NvtxRange nvtx_phase_("fix: double-float phase");
        // FP64-class sweeps in double-float on compact copies of the links and
        // a transform W of the phase (from the identity); at the end W is
        // re-unitarised in FP64 and applied to the FP64 links and transform
        size_t lo_tot = 0, go_tot = 0;
        for (const auto& f : fs) {
            lo_tot += c12_link_chunks(f.g);
            go_tot += c12_gauge_chunks(f.g);
        }
        char* Uh = (char*)scratch_device("fix.df.Uh", 16 * lo_tot, &rc);
        if (rc) return rc;
        char* Ul = (char*)scratch_device("fix.df.Ul", 16 * lo_tot, &rc);
        if (rc) return rc;
        char* Wh = (char*)scratch_device("fix.df.Wh", 16 * go_tot, &rc);
        if (rc) return rc;
        char* Wl = (char*)scratch_device("fix.df.Wl", 16 * go_tot, &rc);
        if (rc) return rc;
        std::vector<FieldDesc> fds(nf);
        size_t lo = 0, go = 0;
        for (int f = 0; f < nf; ++f) {
            const Geom& g = fs[f].g;
            fds[f].U = Uh + 16 * lo;
            fds[f].Ulo = Ul + 16 * lo;
            fds[f].G = Wh + 16 * go;
            fds[f].Glo = Wl + 16 * go;
            fds[f].geo = g;
            fds[f].norm = 1.0 / (9.0 * 8.0 * g.vh);
            lo += c12_link_chunks(g);
            go += c12_gauge_chunks(g);
            if ((rc = launch_to_df((const double*)fs[f].U, fds[f].U, fds[f].Ulo, g, 4, 1, st))) return rc;
            if ((rc = launch_identity_df(fds[f].G, fds[f].Glo, g, 1, st))) return rc;
        }
        rc = run_fix_phase<DoubleFloat>(fds, d_state, h_state, d_hist, hist_len, prm->tol, 1, 1.0, 0,
                                        prm->max_sweeps, prm->check_every, fresh, st);
        if (rc) return rc;
        for (int f = 0; f < nf; ++f)
            if ((rc = launch_handoff(fds[f].G, fds[f].Glo, (double*)fs[f].U, (double*)fs[f].G, fs[f].g, 1, st)))
                return rc;
    } else if (prec == MCG_F64) {
        std::vector<FieldDesc> fds(nf);
        for (int f = 0; f < nf; ++f) {
            fds[f].U = fs[f].U;
            fds[f].G = fs[f].G;
            fds[f].geo = fs[f].g;
            fds[f].norm = 1.0 / (9.0 * 8.0 * fs[f].g.vh);
        }
        rc = run_fix_phase<double>(fds, d_state, h_state, d_hist, hist_len, prm->tol, 1, 1.0, prm->reunit_every,
                                   prm->max_sweeps, prm->check_every, fresh, st, prm->fp64_solve32 != 0);
    } else {
        // FP32 fields: compact copies in, full layout (row 2 rebuilt) out
        std::vector<FieldDesc> fds;
        compact_copies(fds, &rc);
        if (rc) return rc;
        for (int f = 0; f < nf; ++f) {
            if ((rc = launch_to_c12(fs[f].U, MCG_F32, fds[f].U, fs[f].g, 4, 1, st))) return rc;
            if ((rc = launch_to_c12(fs[f].G, MCG_F32, fds[f].G, fs[f].g, 1, 1, st))) return rc;
        }
        rc = run_fix_phase<float>(fds, d_state, h_state, d_hist, hist_len, prm->tol, 1, 1.0, 0, prm->max_sweeps,
                                  prm->check_every, fresh, st);
        if (rc) return rc;
        for (int f = 0; f < nf; ++f) {
            if ((rc = launch_from_c12(fds[f].U, fs[f].U, fs[f].g, 4, 1, st))) return rc;
            if ((rc = launch_from_c12(fds[f].G, fs[f].G, fs[f].g, 1, 1, st))) return rc;
        }
    }
    if (rc) return rc;
    bool all = true;
    for (int f = 0; f < nf; ++f) {
        if (R_out) R_out[f] = h_state[f].R_last;
        if (sweeps_out) sweeps_out[f] = h_state[f].sweep;
        if (sweeps32_out) sweeps32_out[f] = s32[f];
        if (converged_out) converged_out[f] = h_state[f].done == 1;
        all = all && h_state[f].done == 1;
    }
    if (R_hist) {
        MCG_CK(cudaMemcpyAsync(R_hist, d_hist, sizeof(double) * hist_len * (size_t)nf, cudaMemcpyDeviceToHost, st));
        MCG_CK(cudaStreamSynchronize(st));
    }
    return all ? MCG_OK : MCG_NOT_CONVERGED;
}

// uniform batch: nfields fields of lat's dims stored back to back
static int fix_impl(void* U, void* G, const mcg_lattice* lat, const Geom& g, const mcg_params* prm, double* R_out,
                    int* sweeps_out, int* sweeps32_out, double* R_hist, cudaStream_t st, int* converged_out = nullptr,
                    int* restarts_out = nullptr) {
    const size_t eb = elem_bytes(lat->precision);
    std::vector<FieldSpec> fs(lat->nfields);
    for (int f = 0; f < lat->nfields; ++f) {
        fs[f].U = (char*)U + eb * link_elems(g) * f;
        fs[f].G = (char*)G + eb * gauge_elems(g) * f;
        fs[f].g = g;
    }
    return fix_fields(fs, lat->precision, prm, R_out, sweeps_out, sweeps32_out, R_hist, st, converged_out,
                      restarts_out);
}

// validate one entry of an mcg_field array
static int field_spec(const mcg_field& in, int prec, FieldSpec* out) {
    mcg_lattice lat;
    for (int d = 0; d < 4; ++d) lat.dims[d] = in.dims[d];
    lat.nfields = 1;
    lat.precision = prec;
    int rc = check_lat(&lat, &out->g);
    if (rc) return rc;
    if (!in.U || !in.G) return fail(MCG_BAD_ARG, "null field pointer");
    const size_t eb = elem_bytes(prec);
    if (overlap(in.U, eb * link_elems(out->g), in.G, eb * gauge_elems(out->g)))
        return fail(MCG_BAD_ARG, "U and G of a field overlap");
    out->U = in.U;
    out->G = in.G;
    return 0;
}

}  // namespace mcg

using namespace mcg;

// ---------------------------------------------------------------------------
// extern "C" entry points
// ---------------------------------------------------------------------------
extern "C" {

int mcg_version(void) { return 10000; }

const char* mcg_last_error(void) { return g_last_error.c_str(); }

int mcg_release(void) {
    release_all();
    return MCG_OK;
}

int mcg_pack_links(const double* canon, void* U, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!canon || !U) return fail(MCG_BAD_ARG, "null pointer");
    set_error("");
    return launch_pack(canon, U, lat->precision, g, lat->nfields, 0, 0, stream);
}

int mcg_unpack_links(const void* U, double* canon, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!canon || !U) return fail(MCG_BAD_ARG, "null pointer");
    return launch_pack(canon, const_cast<void*>(U), lat->precision, g, lat->nfields, 0, 1, stream);
}

int mcg_pack_gauge(const double* canon, void* G, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!canon || !G) return fail(MCG_BAD_ARG, "null pointer");
    return launch_pack(canon, G, lat->precision, g, lat->nfields, 1, 0, stream);
}

int mcg_unpack_gauge(const void* G, double* canon, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!canon || !G) return fail(MCG_BAD_ARG, "null pointer");
    return launch_pack(canon, const_cast<void*>(G), lat->precision, g, lat->nfields, 1, 1, stream);
}

int mcg_unpack_center(const int8_t* Z, int8_t* canon, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!canon || !Z) return fail(MCG_BAD_ARG, "null pointer");
    return launch_unpack_center(Z, canon, g, lat->nfields, stream);
}

int mcg_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t n_complex, cudaStream_t stream) {
    if (!src || !dst) return fail(MCG_BAD_ARG, "null pointer");
    if ((src_prec != MCG_F64 && src_prec != MCG_F32) || (dst_prec != MCG_F64 && dst_prec != MCG_F32))
        return fail(MCG_BAD_ARG, "bad precision");
    if (overlap(src, n_complex * elem_bytes(src_prec), dst, n_complex * elem_bytes(dst_prec)) && src != dst)
        return fail(MCG_BAD_ARG, "src and dst overlap");
    return launch_convert(src, src_prec, dst, dst_prec, n_complex, stream);
}

int mcg_set_identity_gauge(void* G, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!G) return fail(MCG_BAD_ARG, "null pointer");
    return launch_identity_gauge(G, lat->precision, g, lat->nfields, stream);
}

int mcg_plaquette(const void* U, double* out, const mcg_lattice* lat, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_plaquette");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !out) return fail(MCG_BAD_ARG, "null pointer");
    return compute_plaquette(U, lat->precision, g, lat->nfields, out, stream);
}

int mcg_functional(const void* U, double* R_out, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !R_out) return fail(MCG_BAD_ARG, "null pointer");
    return compute_functional(U, lat->precision, g, lat->nfields, R_out, stream);
}

int mcg_apply_gauge(void* U, const void* G, const mcg_lattice* lat, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_apply_gauge");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !G) return fail(MCG_BAD_ARG, "null pointer");
    const size_t eb = elem_bytes(lat->precision);
    if (overlap(U, eb * link_elems(g) * lat->nfields, G, eb * gauge_elems(g) * lat->nfields))
        return fail(MCG_BAD_ARG, "U and G overlap");
    return launch_apply_gauge(U, G, lat->precision, g, lat->nfields, stream);
}

int mcg_reunitarise(void* M, int which, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!M) return fail(MCG_BAD_ARG, "null pointer");
    if (which != 0 && which != 1) return fail(MCG_BAD_ARG, "which must be 0 (links) or 1 (gauge)");
    return launch_reunitarise(M, which, lat->precision, g, lat->nfields, stream);
}

int mcg_smear(const void* U_in, void* U_out, const mcg_lattice* lat, double rho, double eps, int n,
              cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_smear");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U_in || !U_out) return fail(MCG_BAD_ARG, "null pointer");
    if (n < 0) return fail(MCG_BAD_ARG, "n must be >= 0");
    if (!(std::isfinite(rho) && std::isfinite(eps))) return fail(MCG_BAD_ARG, "rho/eps not finite");
    const size_t bytes = elem_bytes(lat->precision) * link_elems(g) * lat->nfields;
    if (overlap(U_in, bytes, U_out, bytes)) return fail(MCG_BAD_ARG, "U_in and U_out overlap");
    if ((rc = validate_su3(U_in, lat->precision, g, 8, lat->nfields, "mcg_smear: U_in", stream))) return rc;
    return run_smear(U_in, U_out, lat->precision, g, lat->nfields, rho, eps, n, stream);
}

int mcg_fix(void* U, void* G, const mcg_lattice* lat, const mcg_params* params, double* R_out, int* sweeps_out,
            double* R_hist, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_fix");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if (!U || !G) return fail(MCG_BAD_ARG, "null pointer");
    const size_t eb = elem_bytes(lat->precision);
    if (overlap(U, eb * link_elems(g) * lat->nfields, G, eb * gauge_elems(g) * lat->nfields))
        return fail(MCG_BAD_ARG, "U and G overlap");
    if ((rc = validate_su3(U, lat->precision, g, 8, lat->nfields, "mcg_fix: U", stream))) return rc;
    if ((rc = validate_su3(G, lat->precision, g, 2, lat->nfields, "mcg_fix: G", stream))) return rc;
    return fix_impl(U, G, lat, g, params, R_out, sweeps_out, nullptr, R_hist, stream);
}

int mcg_local_solve(const double* A, const double* b, double* a_out, int* fallback_out, int n, int precision,
                    cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_local_solve");
    if (n < 0) return fail(MCG_BAD_ARG, "n must be >= 0");
    if (precision != MCG_F64 && precision != MCG_F32) return fail(MCG_BAD_ARG, "bad precision");
    if (n == 0) return MCG_OK;
    if (!A || !b || !a_out) return fail(MCG_BAD_ARG, "null pointer");
    return launch_local_solve(A, b, a_out, fallback_out, n, precision, stream);
}

int mcg_random_gauge(void* G, const mcg_lattice* lat, unsigned long long seed, unsigned long long seq,
                     cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_random_gauge");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!G) return fail(MCG_BAD_ARG, "null pointer");
    if (lat->precision != MCG_F64) return fail(MCG_BAD_ARG, "mcg_random_gauge takes FP64 fields");
    return launch_random_gauge(G, g, lat->nfields, seed, seq, stream);
}

int mcg_anneal(void* U, void* G, const mcg_lattice* lat, const double* T, int nsweeps, long long first_sweep,
               int nhit, double eps, unsigned long long seed, long long* accepted_out, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_anneal");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (lat->precision != MCG_F64) return fail(MCG_BAD_ARG, "annealing runs on FP64 fields");
    if (lat->nfields > 65535) return fail(MCG_BAD_ARG, "at most 65535 fields per call");
    if (!U || !G || (nsweeps > 0 && !T)) return fail(MCG_BAD_ARG, "null pointer");
    if (nsweeps < 0 || first_sweep < 0) return fail(MCG_BAD_ARG, "nsweeps and first_sweep must be >= 0");
    if (nhit < 1 || nhit > (1 << 20)) return fail(MCG_BAD_ARG, "nhit must be in 1..2^20");
    if (!(eps > 0.0 && eps <= 0.5)) return fail(MCG_BAD_ARG, "eps must be in (0, 0.5]");
    for (int k = 0; k < nsweeps; ++k)
        if (!(T[k] > 0.0)) return fail(MCG_BAD_ARG, "every temperature must be > 0");
    const size_t lb = elem_bytes(MCG_F64) * link_elems(g) * lat->nfields;
    const size_t gb = elem_bytes(MCG_F64) * gauge_elems(g) * lat->nfields;
    if (overlap(U, lb, G, gb)) return fail(MCG_BAD_ARG, "U and G overlap");
    if ((rc = validate_su3(U, MCG_F64, g, 8, lat->nfields, "mcg_anneal: U", stream))) return rc;
    if ((rc = validate_su3(G, MCG_F64, g, 2, lat->nfields, "mcg_anneal: G", stream))) return rc;
    return run_anneal(U, G, g, lat->nfields, T, nsweeps, first_sweep, nhit, eps, seed, accepted_out, stream);
}

int mcg_center_project(const void* U, int8_t* Z, long long* counts, const mcg_lattice* lat, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_center_project");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !Z) return fail(MCG_BAD_ARG, "null pointer");
    // the sector is a function of tr U alone, defined for any finite matrix
    if ((rc = validate_su3(U, lat->precision, g, 8, lat->nfields, "mcg_center_project: U", stream, true))) return rc;
    return compute_center(U, lat->precision, Z, g, lat->nfields, counts, stream);
}

int mcg_vortex_remove(const void* U, const int8_t* Z, void* U_removed, void* U_center, const mcg_lattice* lat,
                      cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_vortex_remove");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !Z) return fail(MCG_BAD_ARG, "null pointer");
    if (!U_removed && !U_center) return fail(MCG_BAD_ARG, "no output requested");
    const size_t bytes = elem_bytes(lat->precision) * link_elems(g) * lat->nfields;
    if (U_center && (overlap(U, bytes, U_center, bytes) || (U_removed && overlap(U_removed, bytes, U_center, bytes))))
        return fail(MCG_BAD_ARG, "U_center overlaps an input or U_removed");
    if (U_removed && U_removed != U && overlap(U, bytes, U_removed, bytes))
        return fail(MCG_BAD_ARG, "U_removed partially overlaps U");
    return launch_vortex_remove(U, Z, U_removed, U_center, lat->precision, g, lat->nfields, stream);
}

int mcg_wilson_loops(const void* U, const mcg_lattice* lat, int Rmax, int Tmax, double* W_out, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_wilson_loops");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !W_out) return fail(MCG_BAD_ARG, "null pointer");
    const int nmin = std::min(g.n[0], std::min(g.n[1], g.n[2]));
    if (Rmax < 1 || Rmax > nmin || Tmax < 1 || Tmax > g.n[3])
        return fail(MCG_BAD_ARG, "need 1 <= Rmax <= smallest spatial extent and 1 <= Tmax <= N_t");
    return compute_wilson_loops(U, lat->precision, g, lat->nfields, Rmax, Tmax, W_out, stream);
}

int mcg_wilson_loops_offaxis(const void* U, const mcg_lattice* lat, const int* vectors, int nvec, int Tmax,
                             double* W_out, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_wilson_loops_offaxis");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !vectors || !W_out) return fail(MCG_BAD_ARG, "null pointer");
    if (nvec < 1) return fail(MCG_BAD_ARG, "nvec must be >= 1");
    if (Tmax < 1 || Tmax > g.n[3]) return fail(MCG_BAD_ARG, "need 1 <= Tmax <= N_t");
    const int nmin = std::min(g.n[0], std::min(g.n[1], g.n[2]));
    for (int v = 0; v < nvec; ++v) {
        int len = 0;
        for (int j = 0; j < 3; ++j) {
            const int c = std::abs(vectors[3 * v + j]);
            if (c >= nmin) return fail(MCG_BAD_ARG, "each |component| must be below the smallest spatial extent");
            len += c;
        }
        if (len < 1 || len > 64) return fail(MCG_BAD_ARG, "path length |r0|+|r1|+|r2| must be in 1..64");
    }
    return compute_wilson_loops_offaxis(U, lat->precision, g, lat->nfields, vectors, nvec, Tmax, W_out, stream);
}

int mcg_precondition_fix(void* U, void* G, int8_t* Z, const mcg_lattice* lat, const mcg_params* params, double rho,
                         double eps, int nsmear, int smear_precision, mcg_precond_result* results,
                         cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_precondition_fix");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if (!U || !G || !results) return fail(MCG_BAD_ARG, "null pointer");
    if (nsmear < 0) return fail(MCG_BAD_ARG, "nsmear must be >= 0");
    if (smear_precision != MCG_F64 && smear_precision != MCG_F32) return fail(MCG_BAD_ARG, "bad smear precision");
    if ((rc = validate_su3(U, lat->precision, g, 8, lat->nfields, "mcg_precondition_fix: U", stream))) return rc;
    const int nf = lat->nfields, prec = lat->precision;
    const size_t le = link_elems(g), ge = gauge_elems(g), eb = elem_bytes(prec);
    std::vector<double> plaq_in(nf), plaq_out(nf), Rs(nf, 0.0), Rf(nf);
    std::vector<int> sw_s(nf, 0), sw_f(nf), sw32_s(nf, 0), sw32_f(nf, 0);
    std::vector<int> conv_s(nf, 1), conv_f(nf, 1), rs_s(nf, 0), rs_f(nf, 0);
    std::vector<long long> counts(7 * (size_t)nf);
    if ((rc = compute_plaquette(U, prec, g, nf, plaq_in.data(), stream))) return rc;
    int status = MCG_OK;
    const double norm = 1.0 / (9.0 * 8.0 * g.vh);
    if ((rc = launch_identity_gauge(G, prec, g, nf, stream))) return rc;
    if (nsmear > 0) {
        // S = smear(U) in the smear precision; the smeared field is then fixed
        // in the field's precision with the caller's schedule (transform W)
        const size_t seb = elem_bytes(smear_precision);
        void* Uc = scratch_device("pre.Uconv", seb * le * nf, &rc);
        if (rc) return rc;
        void* S = scratch_device("pre.S", seb * le * nf, &rc);
        if (rc) return rc;
        void* Sp = scratch_device("pre.Sp", eb * le * nf, &rc);
        if (rc) return rc;
        void* W = scratch_device("pre.W", eb * ge * nf, &rc);
        if (rc) return rc;
        const void* src = U;
        if (smear_precision != prec) {
            if ((rc = launch_convert(U, prec, Uc, smear_precision, le * nf, stream))) return rc;
            src = Uc;
        }
        if ((rc = run_smear(src, S, smear_precision, g, nf, rho, eps, nsmear, stream))) return rc;
        if ((rc = launch_convert(S, smear_precision, Sp, prec, le * nf, stream))) return rc;
        if (smear_precision != prec && (rc = launch_reunitarise(Sp, 0, prec, g, nf, stream))) return rc;
        if ((rc = launch_identity_gauge(W, prec, g, nf, stream))) return rc;
        rc = fix_impl(Sp, W, lat, g, params, Rs.data(), sw_s.data(), sw32_s.data(), nullptr, stream, conv_s.data(),
                      rs_s.data());
        if (rc != MCG_OK && rc != MCG_NOT_CONVERGED) return rc;
        if (rc == MCG_NOT_CONVERGED) status = MCG_NOT_CONVERGED;
        // G <- reunit(W), then U <- U^G (the preconditioning transform)
        MCG_CK(cudaMemcpyAsync(G, W, eb * ge * nf, cudaMemcpyDeviceToDevice, stream));
        if ((rc = launch_reunitarise(G, 1, prec, g, nf, stream))) return rc;
        if ((rc = launch_apply_gauge(U, G, prec, g, nf, stream))) return rc;
    }
    // fix the preconditioned original field, accumulating into G
    rc = fix_impl(U, G, lat, g, params, Rf.data(), sw_f.data(), sw32_f.data(), nullptr, stream, conv_f.data(),
                  rs_f.data());
    if (rc != MCG_OK && rc != MCG_NOT_CONVERGED) return rc;
    if (rc == MCG_NOT_CONVERGED) status = MCG_NOT_CONVERGED;
    int8_t* Zb = Z;
    if (!Zb) {
        Zb = (int8_t*)scratch_device("pre.Z", 8 * (size_t)g.vh * nf, &rc);
        if (rc) return rc;
    }
    if ((rc = compute_center(U, prec, Zb, g, nf, counts.data(), stream))) return rc;
    if ((rc = compute_plaquette(U, prec, g, nf, plaq_out.data(), stream))) return rc;
    for (int f = 0; f < nf; ++f) {
        mcg_precond_result& r = results[f];
        r.V_smeared = Rs[f] * norm;
        r.V_fixed = Rf[f] * norm;
        r.plaquette_in = plaq_in[f];
        r.plaquette_out = plaq_out[f];
        r.vortices = counts[7 * f];
        r.vortex_density = (double)counts[7 * f] / (6.0 * 2.0 * g.vh);
        r.sweeps_smeared = sw_s[f];
        r.sweeps_fixed = sw_f[f];
        r.sweeps_fp32 = sw32_s[f] + sw32_f[f];
        r.status = (conv_s[f] && conv_f[f]) ? MCG_OK : MCG_NOT_CONVERGED;
        r.fp32_restarts = rs_s[f] + rs_f[f];
    }
    return status;
}

long long mcg_kernel_launches(void) { return g_launches.load(); }

int mcg_probe_peaks(double* tflops_out, cudaStream_t stream) {
    if (!tflops_out) return fail(MCG_BAD_ARG, "null pointer");
    return probe_peaks(tflops_out, stream);
}

long long mcg_bounds_violations(int reset) {
#ifdef MCG_CHECK
    cudaDeviceSynchronize();
    const bool r = reset != 0;
    return (long long)(bound_hits_field(r) + bound_hits_observables(r) + bound_hits_smear(r) + bound_hits_sweep(r) +
                       bound_hits_sweep_f32(r) + bound_hits_sweep_df(r));
#else
    (void)reset;
    return -1;
#endif
}

int mcg_phase_stats(double* ms_out, long long* site_updates_out, int reset) {
    if (!ms_out || !site_updates_out) return fail(MCG_BAD_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(g_phase_mu);
    for (int i = 0; i < 2; ++i) {
        ms_out[i] = g_phase_ms[i];
        site_updates_out[i] = g_phase_su[i];
        if (reset) {
            g_phase_ms[i] = 0.0;
            g_phase_su[i] = 0;
        }
    }
    return MCG_OK;
}

int mcg_set_sweep_block(int precision, int threads) {
    if (precision != MCG_F64 && precision != MCG_F32) return fail(MCG_BAD_ARG, "bad precision");
    if (threads != 64 && threads != 128 && !(threads == 256 && precision == MCG_F32))
        return fail(MCG_BAD_ARG, "threads must be 64 or 128 (FP64), 64, 128 or 256 (FP32)");
    set_sweep_block(precision, threads);
    return MCG_OK;
}

int mcg_get_sweep_block(int precision) { return sweep_block(precision); }

int mcg_time_halfsweep(void* U, void* G, const mcg_lattice* lat, int parity, int nreps, int flush_l2, float* ms_out,
                       cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !G || !ms_out) return fail(MCG_BAD_ARG, "null pointer");
    if (lat->nfields != 1) return fail(MCG_BAD_ARG, "mcg_time_halfsweep takes one field");
    if (nreps < 1 || (parity != 0 && parity != 1)) return fail(MCG_BAD_ARG, "nreps >= 1, parity 0 or 1");
    if (lat->precision == MCG_F64) return time_halfsweep<double>(U, G, g, parity, nreps, flush_l2, ms_out, stream);
    // FP32: the kernel runs on the compact working storage; time it on
    // compact copies of U and G (the caller's arrays are left unchanged)
    void* U12 = scratch_device("time.U12", 16 * c12_link_chunks(g), &rc);
    if (rc) return rc;
    void* W12 = scratch_device("time.W12", 16 * c12_gauge_chunks(g), &rc);
    if (rc) return rc;
    if ((rc = launch_to_c12(U, MCG_F32, U12, g, 4, 1, stream))) return rc;
    if ((rc = launch_to_c12(G, MCG_F32, W12, g, 1, 1, stream))) return rc;
    return time_halfsweep<float>(U12, W12, g, parity, nreps, flush_l2, ms_out, stream);
}

int mcg_halfsweep_slab(void* U, void* G, const mcg_lattice* lat, int parity, int t_lo, int t_hi, double* R_out,
                      cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_halfsweep_slab");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !G) return fail(MCG_BAD_ARG, "null pointer");
    if (lat->precision != MCG_F64 || lat->nfields != 1) return fail(MCG_BAD_ARG, "one FP64 field");
    if (parity != 0 && parity != 1) return fail(MCG_BAD_ARG, "parity must be 0 or 1");
    if (t_lo < 0 || t_hi > g.n[3] || t_lo >= t_hi) return fail(MCG_BAD_ARG, "need 0 <= t_lo < t_hi <= N_t");
    if (overlap(U, 16 * link_elems(g), G, 16 * gauge_elems(g))) return fail(MCG_BAD_ARG, "U and G overlap");
    return run_halfsweep_slab(U, G, g, parity, t_lo, t_hi, R_out != nullptr, R_out, stream);
}

int mcg_slab_face(void* U, void* buf, const mcg_lattice* lat, int t, int parity, int to_field, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !buf) return fail(MCG_BAD_ARG, "null pointer");
    if (lat->nfields != 1) return fail(MCG_BAD_ARG, "one field");
    if (parity != 0 && parity != 1) return fail(MCG_BAD_ARG, "parity must be 0 or 1");
    if (to_field != 0 && to_field != 1) return fail(MCG_BAD_ARG, "to_field must be 0 or 1");
    if (t < 0 || t >= g.n[3]) return fail(MCG_BAD_ARG, "need 0 <= t < N_t");
    const size_t eb = elem_bytes(lat->precision);
    // sites of one parity on one layer: a contiguous in-parity range
    // [t * n, (t + 1) * n), n = Nx Ny Nz / 2, in every entry array of U_t
    const size_t n = (size_t)g.n[0] * g.n[1] * g.n[2] / 2;
    if (overlap(U, eb * link_elems(g), buf, eb * 9 * n)) return fail(MCG_BAD_ARG, "buf overlaps U");
    char* face = static_cast<char*>(U) + eb * (((size_t)(3 * 2 + parity) * 9) * g.vh + (size_t)t * n);
    const size_t field_pitch = eb * (size_t)g.vh, width = eb * n;
    cudaError_t e = to_field ? cudaMemcpy2DAsync(face, field_pitch, buf, width, width, 9, cudaMemcpyDeviceToDevice, stream)
                             : cudaMemcpy2DAsync(buf, width, face, field_pitch, width, 9, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "mcg_slab_face copy");
    return MCG_OK;
}

int mcg_precondition_levels(const void* U, void* U_out, void* G_out, int8_t* Z_out, const mcg_lattice* lat,
                            const mcg_params* params, double rho, double eps, const int* nsmear, int nlevels,
                            int smear_precision, mcg_precond_result* results, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_precondition_levels");
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if (lat->nfields != 1) return fail(MCG_BAD_ARG, "mcg_precondition_levels takes one input field");
    if (!U || !U_out || !G_out || !nsmear || !results) return fail(MCG_BAD_ARG, "null pointer");
    if (nlevels < 1) return fail(MCG_BAD_ARG, "nlevels must be >= 1");
    if (smear_precision != MCG_F64 && smear_precision != MCG_F32) return fail(MCG_BAD_ARG, "bad smear precision");
    for (int l = 0; l < nlevels; ++l)
        if (nsmear[l] < 0 || (l > 0 && nsmear[l] < nsmear[l - 1]))
            return fail(MCG_BAD_ARG, "nsmear must be non-negative and non-decreasing");
    if ((rc = validate_su3(U, lat->precision, g, 8, 1, "mcg_precondition_levels: U", stream))) return rc;
    const int prec = lat->precision;
    const size_t le = link_elems(g), ge = gauge_elems(g), eb = elem_bytes(prec), seb = elem_bytes(smear_precision);
    if (overlap(U, eb * le, U_out, eb * le * nlevels)) return fail(MCG_BAD_ARG, "U and U_out overlap");
    const double norm = 1.0 / (9.0 * 8.0 * g.vh);
    double plaq_in = 0;
    if ((rc = compute_plaquette(U, prec, g, 1, &plaq_in, stream))) return rc;
    // smeared levels: one smearing chain, snapshots at each requested level
    std::vector<int> smeared;
    for (int l = 0; l < nlevels; ++l)
        if (nsmear[l] > 0) smeared.push_back(l);
    const int ns = (int)smeared.size();
    std::vector<double> Rs(std::max(ns, 1), 0.0), Rf(nlevels);
    std::vector<int> sw_s(std::max(ns, 1), 0), sw32_s(std::max(ns, 1), 0), sw_f(nlevels), sw32_f(nlevels);
    std::vector<int> conv_s(std::max(ns, 1), 1), conv_f(nlevels, 1);
    std::vector<int> rs_s(std::max(ns, 1), 0), rs_f(nlevels, 0);
    int status = MCG_OK;
    // every level starts from the input field and the identity transform
    for (int l = 0; l < nlevels; ++l)
        MCG_CK(cudaMemcpyAsync((char*)U_out + eb * le * l, U, eb * le, cudaMemcpyDeviceToDevice, stream));
    if ((rc = launch_identity_gauge(G_out, prec, g, nlevels, stream))) return rc;
    void* Sp = nullptr;  // the smeared fields, then their transforms
    void* W = nullptr;
    if (ns > 0) {
        void* cur = scratch_device("lev.cur", seb * le, &rc);
        if (rc) return rc;
        void* tmp = scratch_device("lev.tmp", seb * le, &rc);
        if (rc) return rc;
        Sp = scratch_device("lev.Sp", eb * le * ns, &rc);
        if (rc) return rc;
        W = scratch_device("lev.W", eb * ge * ns, &rc);
        if (rc) return rc;
        if ((rc = launch_convert(U, prec, cur, smear_precision, le, stream))) return rc;
        int done_steps = 0;
        for (int k = 0; k < ns; ++k) {
            const int steps = nsmear[smeared[k]] - done_steps;
            if (steps > 0) {
                if ((rc = run_smear(cur, tmp, smear_precision, g, 1, rho, eps, steps, stream))) return rc;
                std::swap(cur, tmp);
                done_steps += steps;
            }
            if ((rc = launch_convert(cur, smear_precision, (char*)Sp + eb * le * k, prec, le, stream))) return rc;
        }
        if (smear_precision != prec && (rc = launch_reunitarise(Sp, 0, prec, g, ns, stream))) return rc;
        if ((rc = launch_identity_gauge(W, prec, g, ns, stream))) return rc;
    }
    // First batch: the smeared fields and the unsmeared levels (whose fix
    // needs no smearing), so the long fixes run side by side; second batch:
    // the preconditioned copies of the smeared levels.  Per-field arithmetic
    // does not depend on the batch.
    std::vector<FieldSpec> b1, b2;
    std::vector<int> plain_levels;
    for (int k = 0; k < ns; ++k) b1.push_back({(char*)Sp + eb * le * k, (char*)W + eb * ge * k, g});
    for (int l = 0; l < nlevels; ++l)
        if (nsmear[l] == 0) {
            b1.push_back({(char*)U_out + eb * le * l, (char*)G_out + eb * ge * l, g});
            plain_levels.push_back(l);
        }
    {
        const int n1 = (int)b1.size();
        std::vector<double> R1(n1);
        std::vector<int> s1(n1), s321(n1);
        std::vector<int> c1(n1, 1), r1(n1, 0);
        rc = fix_fields(b1, prec, params, R1.data(), s1.data(), s321.data(), nullptr, stream, c1.data(), r1.data());
        if (rc != MCG_OK && rc != MCG_NOT_CONVERGED) return rc;
        if (rc == MCG_NOT_CONVERGED) status = MCG_NOT_CONVERGED;
        for (int k = 0; k < ns; ++k) {
            Rs[k] = R1[k];
            sw_s[k] = s1[k];
            sw32_s[k] = s321[k];
            conv_s[k] = c1[k];
            rs_s[k] = r1[k];
        }
        for (size_t j = 0; j < plain_levels.size(); ++j) {
            const int l = plain_levels[j];
            Rf[l] = R1[ns + j];
            sw_f[l] = s1[ns + j];
            sw32_f[l] = s321[ns + j];
            conv_f[l] = c1[ns + j];
            rs_f[l] = r1[ns + j];
        }
    }
    if (ns > 0) {
        for (int k = 0; k < ns; ++k) {
            char* Gl = (char*)G_out + eb * ge * smeared[k];
            char* Ul = (char*)U_out + eb * le * smeared[k];
            MCG_CK(cudaMemcpyAsync(Gl, (char*)W + eb * ge * k, eb * ge, cudaMemcpyDeviceToDevice, stream));
            if ((rc = launch_reunitarise(Gl, 1, prec, g, 1, stream))) return rc;
            if ((rc = launch_apply_gauge(Ul, Gl, prec, g, 1, stream))) return rc;
            b2.push_back({Ul, Gl, g});
        }
        std::vector<double> R2(ns);
        std::vector<int> s2(ns), s322(ns);
        std::vector<int> c2(ns, 1), r2(ns, 0);
        rc = fix_fields(b2, prec, params, R2.data(), s2.data(), s322.data(), nullptr, stream, c2.data(), r2.data());
        if (rc != MCG_OK && rc != MCG_NOT_CONVERGED) return rc;
        if (rc == MCG_NOT_CONVERGED) status = MCG_NOT_CONVERGED;
        for (int k = 0; k < ns; ++k) {
            Rf[smeared[k]] = R2[k];
            sw_f[smeared[k]] = s2[k];
            sw32_f[smeared[k]] = s322[k];
            conv_f[smeared[k]] = c2[k];
            rs_f[smeared[k]] = r2[k];
        }
    }
    int8_t* Zb = Z_out;
    if (!Zb) {
        Zb = (int8_t*)scratch_device("lev.Z", 8 * (size_t)g.vh * nlevels, &rc);
        if (rc) return rc;
    }
    std::vector<long long> counts(7 * (size_t)nlevels);
    std::vector<double> plaq_out(nlevels);
    if ((rc = compute_center(U_out, prec, Zb, g, nlevels, counts.data(), stream))) return rc;
    if ((rc = compute_plaquette(U_out, prec, g, nlevels, plaq_out.data(), stream))) return rc;
    for (int l = 0; l < nlevels; ++l) {
        mcg_precond_result& r = results[l];
        int k = -1;
        for (int j = 0; j < ns; ++j)
            if (smeared[j] == l) k = j;
        r.V_smeared = k >= 0 ? Rs[k] * norm : 0.0;
        r.sweeps_smeared = k >= 0 ? sw_s[k] : 0;
        r.V_fixed = Rf[l] * norm;
        r.plaquette_in = plaq_in;
        r.plaquette_out = plaq_out[l];
        r.vortices = counts[7 * l];
        r.vortex_density = (double)counts[7 * l] / (6.0 * 2.0 * g.vh);
        r.sweeps_fixed = sw_f[l];
        r.sweeps_fp32 = (k >= 0 ? sw32_s[k] : 0) + sw32_f[l];
        r.status = ((k < 0 || conv_s[k]) && conv_f[l]) ? MCG_OK : MCG_NOT_CONVERGED;
        r.fp32_restarts = (k >= 0 ? rs_s[k] : 0) + rs_f[l];
    }
    return status;
}

int mcg_fix_batch(const mcg_field* fields, int nfields, int precision, const mcg_params* params, double* R_out,
                  int* sweeps_out, cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_fix_batch");
    if (!fields || nfields < 1) return fail(MCG_BAD_ARG, "fields is NULL or nfields < 1");
    if (precision != MCG_F64 && precision != MCG_F32) return fail(MCG_BAD_ARG, "bad precision");
    int rc = check_params(params);
    if (rc) return rc;
    std::vector<FieldSpec> fs(nfields);
    for (int f = 0; f < nfields; ++f)
        if ((rc = field_spec(fields[f], precision, &fs[f]))) return rc;
    for (int f = 0; f < nfields; ++f)
        if ((rc = validate_su3(fs[f].U, precision, fs[f].g, 8, 1, "mcg_fix_batch: U", stream)) ||
            (rc = validate_su3(fs[f].G, precision, fs[f].g, 2, 1, "mcg_fix_batch: G", stream)))
            return rc;
    return fix_fields(fs, precision, params, R_out, sweeps_out, nullptr, nullptr, stream);
}

int mcg_gribov_search(const mcg_field* copies, int ncopies, const int* config_of_copy, int nconfigs, int precision,
                      const mcg_params* params, double* R_out, int* sweeps_out, int* best_copy, double* best_V,
                      cudaStream_t stream) {
    NvtxRange nvtx_range_("mcg_gribov_search");
    if (!copies || ncopies < 1 || !config_of_copy || nconfigs < 1) return fail(MCG_BAD_ARG, "bad copy list");
    if (precision != MCG_F64 && precision != MCG_F32) return fail(MCG_BAD_ARG, "bad precision");
    int rc = check_params(params);
    if (rc) return rc;
    std::vector<FieldSpec> fs(ncopies);
    for (int f = 0; f < ncopies; ++f) {
        if ((rc = field_spec(copies[f], precision, &fs[f]))) return rc;
        if (config_of_copy[f] < 0 || config_of_copy[f] >= nconfigs) return fail(MCG_BAD_ARG, "config index out of range");
    }
    for (int f = 0; f < ncopies; ++f)
        if ((rc = validate_su3(fs[f].U, precision, fs[f].g, 8, 1, "mcg_gribov_search: U", stream)) ||
            (rc = validate_su3(fs[f].G, precision, fs[f].g, 2, 1, "mcg_gribov_search: G", stream)))
            return rc;
    // each copy starts as U^Omega0 with its own random Omega0; the fix then
    // accumulates onto Omega0, so G ends as the total transform of the copy
    for (int f = 0; f < ncopies; ++f)
        if ((rc = launch_apply_gauge(fs[f].U, fs[f].G, precision, fs[f].g, 1, stream))) return rc;
    std::vector<double> R(ncopies);
    std::vector<int> sw(ncopies);
    int st = fix_fields(fs, precision, params, R.data(), sw.data(), nullptr, nullptr, stream);
    if (st != MCG_OK && st != MCG_NOT_CONVERGED) return st;
    std::vector<double> bestV(nconfigs, -1.0);
    std::vector<int> best(nconfigs, -1);
    for (int f = 0; f < ncopies; ++f) {
        const double V = R[f] / (9.0 * 8.0 * fs[f].g.vh);
        const int c = config_of_copy[f];
        if (V > bestV[c]) {  // ties keep the lower copy index
            bestV[c] = V;
            best[c] = f;
        }
        if (R_out) R_out[f] = R[f];
        if (sweeps_out) sweeps_out[f] = sw[f];
    }
    for (int c = 0; c < nconfigs; ++c) {
        if (best_copy) best_copy[c] = best[c];
        if (best_V) best_V[c] = bestV[c];
    }
    return st;
}

int mcg_smear_backward_step(const void* U, const double* Gout, double* Gin, const mcg_lattice* lat, double rho,
                            double eps, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (lat->precision != MCG_F64) return fail(MCG_BAD_ARG, "the smearing backward runs on FP64 fields");
    if (!U || !Gout || !Gin) return fail(MCG_BAD_ARG, "null pointer");
    if (!(std::isfinite(rho) && std::isfinite(eps))) return fail(MCG_BAD_ARG, "rho/eps not finite");
    const size_t bytes = 16 * link_elems(g) * lat->nfields;
    if (overlap(Gin, bytes, Gout, bytes) || overlap(Gin, bytes, U, bytes))
        return fail(MCG_BAD_ARG, "Gin overlaps U or Gout");
    return run_smear_step_backward(U, Gout, Gin, g, lat->nfields, rho, eps, stream);
}

int mcg_functional_matrix_grad(const void* U, double* G, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !G) return fail(MCG_BAD_ARG, "null pointer");
    return run_functional_matrix_grad(U, lat->precision, G, g, lat->nfields, stream);
}

int mcg_grad_R(const void* U, double* grad, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !grad) return fail(MCG_BAD_ARG, "null pointer");
    return run_grad_R(U, lat->precision, grad, g, lat->nfields, stream);
}

int mcg_ascent_step(void* U, void* G, const double* grad, double alpha, const mcg_lattice* lat, cudaStream_t stream) {
    Geom g;
    int rc = check_lat(lat, &g);
    if (rc) return rc;
    if (!U || !G || !grad) return fail(MCG_BAD_ARG, "null pointer");
    if (!std::isfinite(alpha)) return fail(MCG_BAD_ARG, "alpha not finite");
    return run_ascent_step(U, G, grad, alpha, lat->precision, g, lat->nfields, stream);
}

}  // extern "C"
