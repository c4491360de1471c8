// pr_debug.cuh -- checks of the debug build (nvcc -DPR_DEBUG, libpr_debug.so).
//
// compute-sanitizer is not available everywhere this library runs, so the
// debug build carries its own net:
//  - PR_IDX(v, bound, site): every index a kernel loads from a graph array (an
//    in-list source, an out-list target, a frontier entry, a vertex of the
//    permutation) is checked against its bound before it is used.  An index
//    out of range is recorded (the first one with its site, value and bound;
//    all of them counted) and replaced by -1, which every caller treats as "no
//    entry": the access is skipped, nothing outside an array is touched.
//  - After every round of a single solve, the invariants the method keeps
//    (Sec. 3.1, Eq. 4, with the (1-c) reserve) are checked on the device: the
//    mass balance and the residual identity r = p + c P~ s - s, s = x/(1-c)
//    (see k_dbg_invariants in pr_solve.cu).  A deviation beyond the tolerance
//    of the state's arithmetic is recorded the same way.
// A solve whose record holds a failure returns PR_ECHECK.  In a release build
// PR_IDX is the value itself and no check runs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pr.h"

namespace pr {

// check sites (pr_debug_report.first_site)
enum {
    DBG_IN_SRC = 1,      // in-list source id, gathered by a pull round or sweep
    DBG_OUT_DST = 2,     // out-list target id, pushed to by a push round
    DBG_BIN = 3,         // frontier bin entry
    DBG_PERM = 4,        // caller id of an internal vertex (normalisation)
    DBG_TILE_ROW = 5,    // first row of a gather tile
    DBG_SORT_WAIT = 6,   // test hook only: every look-back wait of graph creation's radix sort gives up
    DBG_MASS = 16,       // mass balance after a round (value, bound: deviation and tolerance, x 1e18)
    DBG_IDENTITY = 17,   // residual identity after a round (same units)
};

// the record, one per translation unit and device (every kernel of a unit
// writes the unit's copy; the host reads all units' copies)
struct DbgRec {
    unsigned long long checks;  // invariant checks run
    unsigned long long fails;   // checks that failed
    int32_t site, inject;       // first failing site; the site a test forces to fail (0: none)
    long long value, bound;     // the first failure's value and bound
    double max_mass_dev, max_identity_dev;
};

#ifdef PR_DEBUG
static __device__ DbgRec g_pr_dbg;

__device__ __forceinline__ void dbg_fail(int site, long long value, long long bound) {
    if (atomicAdd(&g_pr_dbg.fails, 1ull) == 0ull) {
        g_pr_dbg.site = site;
        g_pr_dbg.value = value;
        g_pr_dbg.bound = bound;
    }
}

// v if 0 <= v < bound, else -1 (recorded).  A site named by the test hook
// pr_debug_inject sees half its bound, so a valid index above it takes the
// failure path without any invalid access.
__device__ __forceinline__ int dbg_idx(int v, long long bound, int site) {
    const long long b = g_pr_dbg.inject == site ? bound / 2 : bound;
    if (v >= 0 && (long long)v < b) return v;
    dbg_fail(site, v, bound);
    return -1;
}
#define PR_IDX(v, bound, site) ::pr::dbg_idx((v), (bound), (site))
#else
#define PR_IDX(v, bound, site) (v)
#endif

// host side: every translation unit with kernels resets and reads its own
// record (a no-op returning false in a release build)
bool dbg_reset_solve(int inject);
bool dbg_read_solve(DbgRec *out);
bool dbg_reset_batch(int inject);
bool dbg_read_batch(DbgRec *out);
bool dbg_reset_group(int inject);
bool dbg_read_group(DbgRec *out);
bool dbg_reset_sort(int inject);
// the site pr_debug_inject named (0: none)
int dbg_injected();
// around a single or batched solve: clear the records (keeping the injected
// site), then collect them; a failure turns st into PR_ECHECK
void dbg_begin(cudaStream_t s);
pr_status dbg_end(cudaStream_t s, const char *what, pr_status st);

}  // namespace pr
