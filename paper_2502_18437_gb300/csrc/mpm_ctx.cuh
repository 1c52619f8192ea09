// Host-side context of the C ABI (include/mpm.h).
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "mpm_kernels.cuh"

struct mpm_tape;  // recorded trajectory for mpm_backward (mpm_adjoint.cu)

struct mpm_ctx {
    mpm_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    int n_scenes = 0;
    std::vector<int> scene_n, brick_base;  // brick_base has n_scenes + 1 entries
    int total_bricks = 0;
    int cap = 0;
    int total_particles = 0;
    std::vector<mpm::SceneDev> h_scenes;
    std::vector<mpm::RigidDev> h_rigids;  // n_scenes * kMaxRigids
    std::vector<int> rigid_type;          // per slot, MPM_RIGID_NONE when unset
    double h_time = 0.0;                  // scene time (all scenes advance together)

    // device memory
    float* state_mem[2] = {nullptr, nullptr};
    mpm::PState st[2]{};
    int cur = 0;
    mpm::SortBufs sb{};
    std::vector<int> tile_base;  // first scan tile of each scene; n_scenes + 1 entries
    int total_tiles = 0;
    float4* G = nullptr;
    float4* V = nullptr;
    int* brick_epoch = nullptr;
    mpm::SceneDev* d_scenes = nullptr;
    mpm::RigidDev* d_rigids = nullptr;
    double* d_impulse = nullptr;
    unsigned* d_err = nullptr;
    double* d_time = nullptr;
    int* d_epoch = nullptr;
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    void* h_pinned = nullptr;
    size_t pinned_bytes = 0;
    cudaEvent_t ev = nullptr;

    bool keys_valid = false;
    bool scenes_dirty = true;
    // fused substeps leave the next substep's P2G in G: valid for this state and dt
    bool g_pending = false;
    bool g_dirty = false;  // G may hold a pending scatter (must be cleared before a fresh P2G)
    float g_dt = 0.f;
    bool tau_valid = false;  // the stored stress matches the stored F

    // options
    int use_graphs = 1;
    int launch_mode = 0;
    int p2g_chunk = 4 * mpm::kP2GThreads;
    int g2p_threads = 0;  // 0: by the launch's particle count
    int g2p_regs64 = 0;
    int ctas_per_sm = 0;
    int graph_chunk = 32;
    int phase_timing = 0;
    int fused = 0;
    // occupancy (resident CTAs per SM) of each kernel variant on this device, 0 = not asked yet
    int occ_g2p[2][3] = {};
    int occ_p2g[3] = {};
    int occ_grid = 0;
    int occ_grid_plain = 0;
    int occ_fused = 0;
    int occ_p2g_std = 0;
    std::vector<cudaEvent_t> phase_events;  // 5 per timed substep
    size_t phase_used = 0;
    std::map<std::tuple<uint32_t, int, int>, cudaGraphExec_t> graphs;

    mpm_tape* tape = nullptr;
    bool recording = false;
};

namespace mpm {

// helpers shared by the C ABI translation units
int status_from_cuda(cudaError_t e);
int wait_stream(mpm_ctx* c);
StepArgs step_args(mpm_ctx* c, float dt, int s0, int s1, const PState& in, const PState& out);
int enqueue_substep(mpm_ctx* c, float dt, const PState& in, const PState& out, bool need_p2g);
int invalidate_pending(mpm_ctx* c);
int ensure_keys(mpm_ctx* c);
// Zero the brick histogram, the node-brick flags and the tile sums (before keys
// are recomputed from stored positions).
cudaError_t reset_histogram(mpm_ctx* c);
int upload_scenes(mpm_ctx* c);
int ensure_stage(mpm_ctx* c, size_t bytes);
PState state_view(float* base, int cap);
size_t state_bytes(int cap);
void clear_graphs(mpm_ctx* c);

}  // namespace mpm

// tape (mpm_adjoint.cu)
int mpm_tape_record_substep(mpm_ctx* c, float dt);
void mpm_tape_free(mpm_ctx* c);
