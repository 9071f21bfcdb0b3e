// Host-side definition of the case handle and the helpers shared by the
// translation units of the C ABI (single case, batch, server).
#pragma once
#include <string>
#include <vector>

#include "tc_internal.h"
#include <nvtx3/nvToolsExt.h>
#include "../../include/tc.h"

struct HostStencils {
    std::vector<int> start;
    std::vector<double> d0, l1, l2, l4, dwall, dsol;
};

#define TC_MAX_CHUNKS 8

struct tc_handle {
    tc_params prm;
    TcDev d;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<void*> allocs;
    size_t dev_bytes = 0;
    bool need_init = true;
    int phase = 0;                 // next substep (0..2)
    double t = 0.0;
    long long step = 0;
    std::vector<double> r;
    std::vector<double> jac;         // dr/ds of the radial map
    HostStencils S;
    double Ri = 0, Ro = 0;
    cudaStream_t own_stream = nullptr;   // created by the batch / server
    // overlap of the plane and line phases inside a captured step: the
    // azimuthal columns are split into `chunks` groups of z tiles; aux
    // streams 0, 1 run the line kernel of alternate chunks, 2 the mean flow,
    // 3 the next substep's z inverse (0 chunks: chosen from the shape)
    int chunks = 0;                // set by tc_set_tiles (0: automatic)
    int chunks_auto = 0;           // chosen by timing the first steps (0: not yet)
    bool pipe_ready = false;
    cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t evz[TC_MAX_CHUNKS] = {}, evl[TC_MAX_CHUNKS] = {}, evm = nullptr, evj[4] = {};
    // deferred RK memory (double-float and mixed forms): the implicit part of
    // substep k's RK memory runs on srk beside the theta rows of substep k+1
    // (rk_defer: -1 chosen by timing, 0 off, 1 on; rk_defer_auto: the
    // timed choice).  tc_step then runs graph_first, graph_next (which
    // starts the previous step's last RK memory beside its own theta rows)
    // and completes the last one after the final step; `graph` is the
    // self-contained step (the server launches it one step at a time).
    cudaStream_t srk = nullptr;
    cudaEvent_t evrk0 = nullptr, evrk1 = nullptr;
    int rk_defer = -1, rk_defer_auto = -1;
    cudaGraphExec_t graph_first = nullptr, graph_next = nullptr;
    // this rank's share of a case split across ranks (tc_split_set): radial
    // planes [r0, r1) of the plane phase, azimuthal columns [j0, j1) of the
    // line phase, and the products of its planes [TC_NPROD][r1-r0][Nz][Nh]
    bool split = false;
    int split_r0 = 0, split_r1 = 0, split_j0 = 0, split_j1 = 0;
    void* prod_slab = nullptr;
};

namespace tcx {
// NVTX range over one API call (visible in Nsight timelines; free without a
// tool attached)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
void set_err(const std::string& s);
int ensure_init(tc_handle* h);                 // H_1 and u, w of the current state
// the kernels of one step (lead / trail: see the deferred RK memory above)
void launch_step(tc_handle* h, cudaStream_t s, bool lead, bool trail);
int ensure_graph(tc_handle* h);
void drop_graphs(tc_handle* h);                // the captured steps (after a change of launch shapes)
bool defer_rk(const tc_handle* h);            // deferred RK memory in the captured steps
int prepare_pipeline(tc_handle* h);           // aux streams and events (before any capture)
int pipeline_chunks(const tc_handle* h);      // column groups of the overlapped step (1: none)
bool chunks_valid(const tc_handle* h, int c);
void release_pipeline(tc_handle* h);
int check_flags(tc_handle* h);
size_t estimate_device_bytes(const tc_params& p);
int validate(const tc_params* p);
}  // namespace tcx
