// Host-side query of the reflector store's order (no GPU needed).
//
// band_to_bidiag_vectors keeps, for every row-bulge of the reduction, its
// right and left reflectors: row-bulge k holds slots 2k (right) and 2k + 1
// (left).  The kernels that generate a reflector compute k in closed form,
// the stage's base (row-bulges of the earlier stages) plus steps_before(R)
// plus s; the back-transformation (Q and P for the singular vectors that
// Section VII leaves to future work: the products of the stored reflectors
// in the order of the sequential schedule) walks the store with a running
// counter in stage, sweep, step order.  This
// entry point evaluates the closed form exactly as the launch code does, so
// the host tests can check it against the counter order.
#include <algorithm>

#include "../../include/band_bidiag.h"
// The header defines the device-side bounded wait as a plain (non-inline)
// function for the reduction's translation unit; this unit never calls it,
// and the rename keeps the two object files' symbols apart at link time.
#define wait_at_least wait_at_least_unused_in_refl_index
#include "bb_device.cuh"
#undef wait_at_least

extern "C" int bb_reflector_index(int64_t n64, int64_t b64, int tw, int stage, int64_t R, int64_t s,
                                  int64_t* k_out)
{
    if (n64 < 1 || b64 < 0 || tw < 1 || stage < 0 || n64 >= bb::PROG_STAGE || !k_out) return BB_ERR_ARG;
    const int n = (int)n64;
    int bw = (int)std::min<int64_t>(b64, std::max<int64_t>(n64 - 1, 0));
    int64_t base = 0;
    for (int st = 0; st < stage && bw > 1; ++st) {
        const int d = std::min(tw, bw - 1);
        base += bb::steps_before(n, bw, d, n);
        bw -= d;
    }
    if (bw <= 1 || R < 0 || R > n - 2 || s < 0) return BB_ERR_ARG;
    const int d = std::min(tw, bw - 1);
    const int64_t c0 = R + (bw - d);
    const int64_t ns = c0 >= n - 1 ? 0 : (n - 2 - c0) / bw + 1;
    if (s >= ns) return BB_ERR_ARG;
    *k_out = base + bb::steps_before(n, bw, d, R) + s;
    return BB_OK;
}
