// pr_group.cuh -- column groups (K solves on one graph sharing each gather):
// the device view of a group and the launchers, for the request server.
#pragma once

#include "pr_internal.cuh"

namespace pr {

struct Ctl;

// Device view of one group.  x, r: [n][K] state values; w[0], w[1]: [n_nd][K]
// pending pushes, w[launch_id & 1] written by launch launch_id.  ctl[k] is the
// control block of the solve in column k (nullptr: free); join[k] is the launch
// id of that column's first round (-1: none).
struct GroupDev {
    void *x, *r;
    void *w[2];
    Ctl *ctl[8];
    int32_t join[8];
    double *slot_r;  // [kMaxBlocks][K] per-block column partials (8-byte slots)
    long long *slot_f, *slot_e;
    uint32_t *ticket;
};

int group_columns(int fmt);                          // fmt 0: float state (8 columns); 1: double-float (4)
size_t group_bytes(const pr_graph *g, int fmt);      // device bytes of one group on g
void group_layout(const pr_graph *g, int fmt, void *base, GroupDev &D);  // carve a block of group_bytes
pr_status group_round(const pr_graph *g, const GroupDev &D, int fmt, int32_t launch_id, cudaStream_t s);
pr_status group_load(const pr_graph *g, const GroupDev &D, int fmt, int col, const void *x, const void *r,
                     cudaStream_t s);
pr_status group_extract(const pr_graph *g, const GroupDev &D, int fmt, int col, void *x, void *r, cudaStream_t s);

}  // namespace pr
