// Feeds residual samples to the run-to-steady stall rule (csrc/lbc_stall.h).
// stdin: window, then lines "done residual" in increasing done. stdout: the done of the
// first sample at which the rule reports a stall, or -1.
#include <cstdio>

#include "lbc_stall.h"

int main()
{
    long window = 0;
    if (std::scanf("%ld", &window) != 1 || window <= 0) return 2;
    lbc::StallTrack t;
    long done = 0;
    double r = 0.0;
    int got;
    while ((got = std::scanf("%ld %lf", &done, &r)) == 2)
        if (lbc::stall_sample(t, done, r, window)) {
            std::printf("%ld\n", done);
            return 0;
        }
    if (got != EOF) return 3;   // a line that is not "done residual"
    std::printf("-1\n");
    return 0;
}
