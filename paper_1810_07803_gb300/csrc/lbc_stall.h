// Run-to-steady stall rule (lbc_set_stall_window): host logic only, no CUDA.
#pragma once
#include <algorithm>
#include <cmath>
#include <deque>
#include <utility>

namespace lbc {

// Fraction of the earlier low that a window's low must undercut for the instance to go on.
constexpr double kStallGain = 0.99;

// One instance's residual history. Residuals are sampled at the end of each group of steps;
// the instance has stalled once no sample of its last `window` steps sets a new low, by 1 %,
// against the samples before them. A residual that still contracts keeps setting lows however
// slowly it contracts (any rate^window < 0.99 passes); one that has reached the rounding noise
// of its arithmetic (about 1e-9 for an FP32 state) wanders about a level and soon stops.
struct StallTrack {
    std::deque<std::pair<long, double>> recent;   // (steps done, residual) within the window
    double best_before = INFINITY;                // lowest residual sampled before it
    bool stalled = false;
};

// Adds the sample (done, r), done increasing; true if the instance has stalled. window > 0.
inline bool stall_sample(StallTrack &t, long done, double r, long window)
{
    t.recent.emplace_back(done, r);
    while (t.recent.front().first <= done - window) {   // ends: the new sample stays (window > 0)
        t.best_before = std::min(t.best_before, t.recent.front().second);
        t.recent.pop_front();
    }
    if (!(t.best_before < INFINITY)) return false;     // less than one window sampled yet
    double best = INFINITY;
    for (const auto &smp : t.recent) best = std::min(best, smp.second);
    return !(best < kStallGain * t.best_before);
}

}  // namespace lbc
