// Host-side definition of the case handle and the helpers shared by the
// translation units of the C ABI (single case, batch, server).
#pragma once
#include <string>
#include <vector>

#include "tc_internal.h"
#include "../../include/tc.h"

struct HostStencils {
    std::vector<int> start;
    std::vector<double> d0, l1, l2, l4, dwall, dsol;
};

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
};

namespace tcx {
void set_err(const std::string& s);
int ensure_init(tc_handle* h);                 // H_1 and u, w of the current state
void launch_step(tc_handle* h, cudaStream_t s);  // the 15 kernels of one step
int ensure_graph(tc_handle* h);
int check_flags(tc_handle* h);
size_t estimate_device_bytes(const tc_params& p);
int validate(const tc_params* p);
}  // namespace tcx
