// klb_handle.h -- the state behind a klb_t handle (internal to the library;
// shared by the single-grid C ABI and the batch engine).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/klb.h"
#include <nvtx3/nvToolsExt.h>
#include "klb_launch.h"

using fdlb::Geom;
using fdlb::InstDesc;
using fdlb::StepConst;

struct klb {  // state of one grid
    klb_params p{};
    Geom g{};
    size_t esize = 0;             // bytes per element of f
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;                  // buffer holding the current state
    CUtensorMap map[2];
    StepConst<float> cf{};
    StepConst<double> cd{};
    double* fields_dev = nullptr; // 4 * nx * ny doubles of staging for host fields
    double* fdense_dev = nullptr; // 19 * nx * ny doubles of staging for host f (lazy)
    double* diag_ring = nullptr;  // [cap][7]
    double* diag_partials = nullptr;
    int nparts = 0;
    int cap = 0;
    int* err_dev = nullptr;
    int64_t steps = 0;
    bool pending_sample = false;
    bool initialized = false;
    bool broken = false;          // a failed tile-shape rollback left maps and descriptors inconsistent
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t launches = 0;
    long long spin_limit = fdlb::kDefaultSpin;
    int inject = 0;
    int variant = 0;  // FP32 tile shape (see klb_set_variant)
    InstDesc* descs_dev = nullptr;   // FP32: descriptors of the state in buf[0] / buf[1] (2 entries)
    int ntiles = 0;                  // FP32: tiles of one launch (current variant)
    long long* nsamp_dev = nullptr;  // samples taken (device counter; the finalize kernel advances it)
    // FP32 WENO5: runs of graph_steps steps replayed from CUDA graphs, by
    // starting parity and whether the starting state's sample is due
    int graph_steps = 0;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t graph_launches[2][2] = {{0, 0}, {0, 0}};
    bool use_graph = true;
    std::string err;
};

namespace fdlb {

// Tracing: an NVTX range (visible to Nsight tools; no cost without one) over
// one call of the library's public API.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
// the step constants of a problem statement, in either arithmetic type
void step_constants(const klb_params& p, StepConst<float>& c);
void step_constants(const klb_params& p, StepConst<double>& c);
// helpers of klb_capi.cu used by the batch engine
int handle_fail(klb_t* h, int code, const std::string& msg);
int handle_upload_descs(klb_t* h);  // (re)build the FP32 descriptors and the tile count
void handle_drop_graphs(klb_t* h);  // forget the captured step graphs (their launches changed)
// TMA map of a state buffer of the handle's layout (x: pitch, y: rows with
// ghosts, z: 19 planes) with a box of bx x by x bz elements
int encode_state_map(klb_t* h, const void* base, unsigned bx, unsigned by, unsigned bz, CUtensorMap* map);
void handle_after_step(klb_t* h);   // advance the step counter and the parity
}  // namespace fdlb
