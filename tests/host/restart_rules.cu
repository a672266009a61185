// Host-side rules of the FP32-phase restarts (mcg_internal.h), run on the CPU:
// the creep test and the over-relaxation sequence.  Prints one line per case
// ("name ok" or "name FAIL ...") and exits non-zero on a failure.
#include <cmath>
#include <cstdio>
#include <vector>

#include "mcg_internal.h"

static int failures = 0;
static void check(bool ok, const char* name) {
    std::printf("%s %s\n", name, ok ? "ok" : "FAIL");
    if (!ok) ++failures;
}

int main() {
    using mcg::creeping;
    using mcg::restart_omega;
    const double lo = 1e-10, hi = 1e-9;
    // a flat creep at 2e-10 per sweep: restart
    std::vector<double> flat(120, 2e-10);
    check(creeping(flat.data(), 120, lo, hi), "flat_creep");
    // a slow decay 1/k inside the band, from 3.2e-10 to 2.6e-10: still creeping
    std::vector<double> slow(120);
    for (int i = 0; i < 120; ++i) slow[i] = 3.2e-10 * 1000.0 / (1000.0 + 2.0 * i);
    check(creeping(slow.data(), 120, lo, hi), "slow_decay_creeps");
    // a converging fix: exponential decay by more than half over the window
    std::vector<double> conv(120);
    for (int i = 0; i < 120; ++i) conv[i] = 9e-10 * std::exp(-i / 60.0);
    for (int i = 0; i < 120; ++i) conv[i] = std::fmax(conv[i], 1.05e-10);
    check(!creeping(conv.data(), 120, lo, hi), "decay_is_not_creep");
    // one chunk outside the band (a spike, or the drift floor): no restart
    std::vector<double> spike = flat;
    spike[60] = 1.2e-5;
    check(!creeping(spike.data(), 120, lo, hi), "spike_is_not_creep");
    std::vector<double> floor_ = flat;
    floor_[119] = 3e-11;
    check(!creeping(floor_.data(), 120, lo, hi), "floor_is_not_creep");
    // a negative chunk (R fell: an over-relaxed step) is outside the band
    std::vector<double> neg = flat;
    neg[0] = -1e-10;
    check(!creeping(neg.data(), 120, lo, hi), "negative_is_not_creep");
    // NaN never creeps; too few chunks never creep
    std::vector<double> nan = flat;
    nan[5] = std::nan("");
    check(!creeping(nan.data(), 120, lo, hi), "nan_is_not_creep");
    check(!creeping(flat.data(), 3, lo, hi), "short_window");
    // the over-relaxation of the k-th restart: omega, omega - d, omega + d, omega - 2d, ...
    const double w = 1.9, d = 0.03;
    const double want[6] = {1.9, 1.87, 1.93, 1.84, 1.96, 1.81};
    bool seq = true;
    for (int k = 0; k < 6; ++k) seq = seq && std::fabs(restart_omega(w, d, k) - want[k]) < 1e-12;
    check(seq, "omega_sequence");
    // d = 0.15 from 1.9: 1.75, then 2.05 (outside (0, 2): no further restart)
    check(std::fabs(restart_omega(1.9, 0.15, 1) - 1.75) < 1e-12 && restart_omega(1.9, 0.15, 2) >= 2.0,
          "omega_leaves_range");
    return failures ? 1 : 0;
}
