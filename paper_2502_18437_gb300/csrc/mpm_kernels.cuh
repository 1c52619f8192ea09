// Kernel parameter blocks and host-side launchers of the forward substep.
#pragma once

#include "mpm_device.cuh"

namespace mpm {

struct Range {
    int s0, s1;     // scene range [s0, s1)
    int bb0, nbr;   // global brick range [bb0, bb0 + nbr)
    int t0, nt;     // scan tile range [t0, t0 + nt)
    int p0, np;     // particle range [p0, p0 + np)
};

struct SortBufs {
    int* key;       // [cap] brick x 64 + base cell of each stored particle (next substep)
    int* rank;      // [cap] rank of the particle within its brick
    int* perm;      // [cap] sorted slot -> storage index
    unsigned char* scell; // [cap] sorted slot -> base cell inside its brick (the key's low 6 bits)
    int* cnt;       // [bricks] particles per brick (next substep)
    int* nflag;     // [bricks] node brick touched by a particle brick's stencil (set by the
                    // key producers, read by the scan, cleared by k_grid_clear)
    int* off;       // [bricks] first slot of each active brick
    int* act_brick; // [bricks] active particle bricks
    int* act_start;
    int* act_count;
    int* act_scene;
    int* nact_brick;// [bricks] active node bricks
    int* nact_scene;
    int* counters;  // [CTR_COUNT]
    int4* tile_sum; // [tiles] per scan tile (particles, active particle bricks, active node
                    // bricks, particle bricks of at least kBigBrick particles) of the
                    // next substep, added up by the key producers, read by the scan
                    // and cleared by the scatter
    int tile_shift; // log2 of the bricks per scan tile
};

struct StepArgs {
    Range r;
    SortBufs sb;
    const SceneDev* scenes;
    const RigidDev* rigids;      // [n_scenes * kMaxRigids]
    double* impulse;             // [n_scenes * kMaxRigids * 6]
    double* t_scene;             // [n_scenes] scene clocks
    int* epoch;                  // [n_scenes] substep counters
    int* brick_epoch;            // [bricks] substep of the last grid update of a node brick
    unsigned* err;               // [n_scenes]
    float4* G;                   // P2G accumulator (m, mv)
    float4* V;                   // node (v, m)
    PState in, out;
    int cap;
    float dt;
    float gravity[3];
    int bound, floor_sticky;
    int model, plasticity;
    float yield_stress;
    int persistent_ctas;         // CTAs of the persistent G2P kernel
    int p2g_ctas, grid_ctas;     // CTAs of the persistent P2G and grid kernels
    int grid_plain_ctas;         // CTAs of the grid kernel of launches without rigids
    int fused_ctas;              // CTAs of the fused G2P + P2G kernel
    int p2g_chunk, g2p_threads, g2p_regs64;
    int tau_valid;               // P2G reads the stored stress (else recomputes it from F)
    int any_rigid;               // some scene of the range has a rigid (contact in the grid update)
    int rigid_ext;               // some scene of the range has an arc or a mesh slicer
    int any_solid;               // some scene of the range has a sphere or a box (particle push-out)
    int cell_order;              // P2G rewrites each pass's permutation slots in cell order
    int solver;                  // MPM_SOLVER_*
    float pb_beta;               // PB-MPM constraint blend
};

constexpr int kStateFloats = 32;  // x3 v3 C9 F9 tau6 mu lam (+ int id)
constexpr int kP2GThreads = 192;  // 64 cells x 3 node slices
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;  // bricks per pass of a scan CTA
constexpr int kScatterPer = 4;  // particles per thread of the counting-sort scatter
// Particle bricks of at least this many particles come first in the active list,
// so the persistent transfer kernels end on small bricks (a shorter tail)
constexpr int kBigBrick = 256;

cudaError_t launch_prepare(const StepArgs& a, const PState& st, cudaStream_t s);
cudaError_t launch_sort(const StepArgs& a, cudaStream_t s, bool write_perm = true);
cudaError_t launch_p2g(const StepArgs& a, cudaStream_t s);
cudaError_t prepare_p2g();  // shared-memory opt-in of the P2G variants (once per device, before any launch)
cudaError_t launch_grid(const StepArgs& a, cudaStream_t s);
cudaError_t launch_g2p(const StepArgs& a, cudaStream_t s);
cudaError_t launch_p2g_std(const StepArgs& a, cudaStream_t s);  // standard MPM P2G
cudaError_t launch_g2p_vc(const StepArgs& a, cudaStream_t s);   // PB-MPM cycle G2P (v, C in place)
int occupancy_p2g_std();
cudaError_t launch_g2p2g(const StepArgs& a, cudaStream_t s);
int occupancy_g2p2g();
int occupancy_grid();
int occupancy_grid_plain();

// state I/O helpers
cudaError_t launch_gather_field(const PState& st, int cap, int p0, int np, int field, void* dst,
                                cudaStream_t s);
cudaError_t launch_init_particles(const PState& st, int cap, int p_at, int n, int id0, const float* x,
                                  const float* v, const float* E, const float* nu, float E0, float nu0,
                                  cudaStream_t s);
cudaError_t launch_permute_to_id(const PState& src, const PState& dst, int cap, int p0, int np,
                                 cudaStream_t s);
cudaError_t launch_scatter_field(const PState& st, int cap, int p0, int np, int field, const float* src,
                                 cudaStream_t s);
// x, v, C, F (null: not moved) of one scene as host-mapped arrays in particle-id order
struct HostFields {
    float* f[4];
};
// inv[id] = slot of the scene's particle with that id (np entries)
cudaError_t launch_id_inverse(const PState& st, int p0, int np, int* inv, cudaStream_t s);
// state fields <-> host-mapped arrays in one pass (to_host: state -> host)
cudaError_t launch_fields_host(const PState& st, int cap, int p0, int np, const int* inv, const HostFields& h,
                               bool to_host, cudaStream_t s);
cudaError_t launch_read_grid(const float4* V, const int* brick_epoch, const int* epoch, const SceneDev* scenes,
                             int scene, int n, int brick_base, float* dst, cudaStream_t s);
int occupancy_p2g(int chunk);
int occupancy_g2p(int threads, int regs64);

}  // namespace mpm
