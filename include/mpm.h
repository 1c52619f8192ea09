/*
 * mpm.h - C ABI of the GB300-native MLS-MPM substep library.
 *
 * The library advances soft bodies discretised as material points with the
 * moving-least-squares MPM of arXiv 2502.18437 (CRESSim-MPM), Sec. III-B,
 * Algorithm 1: particle-to-grid transfer (Eq. 1, Eq. 8), grid update with
 * gravity (Eq. 3), contact against rigid surgical geometries (Sec. IV, Eq. 11,
 * Eq. 12) and domain walls, grid-to-particle transfer (Eq. 4, Eq. 9) and the
 * deformation-gradient update (Eq. 10) with the constitutive law (Eq. 6).
 * The call pattern follows the paper's object model (Sec. V-A): an
 * asynchronous "advance" (mpm_substep) and a blocking "fetch results"
 * (mpm_read_state), with a factory that creates particle objects and rigid
 * shapes (mpm_add_particles, mpm_set_rigid).
 *
 * Conventions shared by every call
 *  - Units are SI.  Each scene's domain is the unit cube [0,1)^3 on a grid of
 *    n^3 nodes, dx = 1/n, node (i,j,k) at (i,j,k)*dx.  n is a multiple of 4.
 *  - 3-vectors are stored as 3 consecutive floats per particle ((N,3) row
 *    major); 3x3 matrices as 9 consecutive floats, row major ((N,3,3)).
 *  - `mem` says where a caller buffer lives: MPM_MEM_HOST (any host memory)
 *    or MPM_MEM_DEVICE (device memory of the context's GPU, e.g. a torch
 *    tensor's data_ptr()).  The library never frees caller memory and copies
 *    every input before the call returns; output buffers are owned by the
 *    caller.
 *  - Every call returns MPM_OK (0) or a negative MPM_ERR_* code; no call traps
 *    the GPU, and every wait is bounded by mpm_config.timeout_ms.
 *  - Errors found on the device (a particle leaving the grid, a non-finite
 *    value, an inverted element where the law has no answer) are recorded per
 *    scene, are sticky until mpm_destroy, and are returned by the blocking
 *    calls (mpm_read_state, mpm_get_error).
 *  - A context is used from one host thread at a time; its work is ordered on
 *    the CUDA stream given to mpm_create.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MPM_OK 0
#define MPM_ERR_INVALID_ARGUMENT (-1) /* bad pointer, size, index or option      */
#define MPM_ERR_OUT_OF_MEMORY (-2)    /* a device or pinned host allocation failed */
#define MPM_ERR_CUDA (-3)             /* a CUDA runtime call failed              */
#define MPM_ERR_OUT_OF_DOMAIN (-4)    /* a particle's stencil left its scene's grid */
#define MPM_ERR_NONFINITE (-5)        /* a particle position/velocity/F became inf/NaN */
#define MPM_ERR_INVERTED (-6)         /* det F <= 0 where the law needs ln J     */
#define MPM_ERR_CAPACITY (-7)         /* more particles than max_particles       */
#define MPM_ERR_TIMEOUT (-8)          /* a bounded wait ran out                  */
#define MPM_ERR_STATE (-9)            /* call out of order (e.g. no tape recorded) */
#define MPM_ERR_INTERNAL (-10)        /* a device-side consistency check failed      */

/* device error bits reported by mpm_get_error */
#define MPM_EBIT_OUT_OF_DOMAIN 1u
#define MPM_EBIT_NONFINITE 2u
#define MPM_EBIT_INVERTED 4u
#define MPM_EBIT_TIMEOUT 8u
#define MPM_EBIT_INTERNAL 16u /* sort bookkeeping inconsistent: the substep's work was skipped */

/* ---- enumerations ---------------------------------------------------- */
enum { MPM_MEM_HOST = 0, MPM_MEM_DEVICE = 1 };
enum { MPM_FIXED_COROTATED = 0, MPM_NEO_HOOKEAN = 1 };
enum { MPM_PLASTIC_NONE = 0, MPM_PLASTIC_VON_MISES = 1 };
/* Solvers (Sec. III).  MLS: APIC-style MLS-MPM, Algorithm 1 (Sec. III-B).
 * STANDARD: PIC transfers with the internal force -V sigma grad phi (Eq. 1-6,
 * Sec. III-A); C then holds the velocity gradient L of the F update.
 * PB: position-based MPM (Sec. III-C): each substep runs pb_iterations cycles
 * of the co-rotational constraint in P2G, the APIC transfers and the grid
 * update at fixed positions, then integrates x and F; gravity enters once per
 * substep, contact and walls act in every cycle (their momentum is booked to
 * the rigids in every cycle), plasticity and mpm_backward are not available. */
enum { MPM_SOLVER_MLS = 0, MPM_SOLVER_STANDARD = 1, MPM_SOLVER_PB = 2 };
enum { MPM_SPHERE = 0, MPM_BOX = 1, MPM_QUAD_SLICER = 2, MPM_SEGMENTS = 3, MPM_ARC = 4, MPM_MESH_SLICER = 5,
       MPM_RIGID_NONE = -1 };

#define MPM_MAX_SEGMENT_POINTS 64
#define MPM_MAX_MESH_TRIANGLES 64
#define MPM_MAX_SPINE_POINTS 16
#define MPM_MAX_RIGIDS 8 /* per scene */

/* fields of mpm_read_state / mpm_write_state (bitmask; buffers in bit order) */
#define MPM_FIELD_X 1u        /* float (N,3) positions                          */
#define MPM_FIELD_V 2u        /* float (N,3) velocities                         */
#define MPM_FIELD_C 4u        /* float (N,3,3) affine velocity matrix (Eq. 9)   */
#define MPM_FIELD_F 8u        /* float (N,3,3) deformation gradient (Eq. 10)    */
#define MPM_FIELD_ORDER 16u   /* read only: int32 (N) particle ids in storage order */
#define MPM_FIELD_IMPULSE 32u /* read only: double (MPM_MAX_RIGIDS,6) momentum given
                                 to each rigid (linear, angular about its centre)
                                 since the previous read of this field; reading resets it */

/* options of mpm_set_option */
enum {
    MPM_OPT_USE_GRAPHS = 1,     /* 0/1: replay substeps from captured CUDA graphs   */
    MPM_OPT_LAUNCH_MODE = 2,    /* 0: one launch per phase over all scenes;
                                   1: one launch per phase per scene (looped)       */
    MPM_OPT_P2G_THREADS = 3,    /* threads per CTA of the P2G kernel: fixed at 192
                                   (64 cells x 3 node slices); other values rejected */
    MPM_OPT_G2P_THREADS = 4,    /* threads per CTA of the G2P kernel: 128 / 256 / 512,
                                   or 0 (default): 256 for launches of fewer than
                                   524,288 particles, else 128 (reads back the shape
                                   of a launch over all scenes)                      */
    MPM_OPT_CTAS_PER_SM = 5,    /* persistent CTAs per SM for P2G/G2P (0 = occupancy max) */
    MPM_OPT_GRAPH_CHUNK = 6,    /* most substeps captured per graph (1..64, default 32):
                                   a call of k substeps replays ceil(k/chunk) graphs */
    MPM_OPT_PHASE_TIMING = 7,   /* 0/1: record CUDA events around each phase of every
                                   substep (forces direct launches); see mpm_phase_stats */
    MPM_OPT_P2G_CHUNK = 8,      /* particles staged per pass of the P2G kernel: 384,
                                   576 or 768 (default)                             */
    MPM_OPT_FUSED = 9,          /* 1: fuse each substep's G2P with the next substep's
                                   P2G; 0 (default): separate P2G and G2P kernels */
    MPM_OPT_G2P_REGS64 = 10     /* 1: G2P variant limited to 64 registers (more
                                   resident warps); 0 (default): the larger budget
                                   (72 registers at 128 threads, 80 at 256, 112
                                   at 512)                                          */
};

/* ---- configuration --------------------------------------------------- */
typedef struct {
    int32_t n_scenes;            /* independent scenes advanced together (>= 1)       */
    int32_t grid_n;              /* nodes per dimension of every scene (multiple of 4,
                                    8..1024) unless scene_grid_n is given            */
    const int32_t* scene_grid_n; /* optional host array [n_scenes] of per-scene n     */
    int64_t max_particles;       /* capacity summed over scenes                       */
    int32_t model;               /* MPM_FIXED_COROTATED or MPM_NEO_HOOKEAN            */
    int32_t plasticity;          /* MPM_PLASTIC_NONE or MPM_PLASTIC_VON_MISES         */
    float yield_stress;          /* von Mises yield on the Kirchhoff stress (Pa)      */
    float gravity[3];            /* m/s^2                                             */
    int32_t bound;               /* wall thickness in nodes at every face (>= 0)      */
    int32_t floor_sticky;        /* 1: the y-low wall is sticky; 0: it slips           */
    int32_t timeout_ms;          /* bound on every blocking wait (<= 0: 10000)        */
    int32_t tape_checkpoint_every; /* > 0 enables mpm_tape_begin/mpm_backward; the
                                      tape stores a checkpoint every this many substeps */
    int32_t tape_max_substeps;   /* longest recordable tape (substeps)               */
    int32_t solver;              /* MPM_SOLVER_MLS (0, default), MPM_SOLVER_STANDARD or
                                    MPM_SOLVER_PB (Sec. III: the paper's three solvers) */
    int32_t pb_iterations;       /* PB-MPM: P2G-G2P cycles per step (0: 10)           */
    float pb_beta;               /* PB-MPM: blend beta in [0,1] of the co-rotational
                                    constraint (1: rotation only, stiffest)          */
    int32_t reserved[4];         /* zero */
} mpm_config;

/* A rigid body (Sec. IV).  Body frame -> world frame by the unit quaternion
 * quat = (w,x,y,z) and the centre; the body moves kinematically with vel and
 * omega (world frame) from the moment it is set, and the host updates it
 * between steps (Sec. V-C).  Contact regions, with margin the fattening of
 * the region:
 *  MPM_SPHERE      radius; signed distance < margin
 *  MPM_BOX         half[3] half extents; signed distance < margin
 *  MPM_QUAD_SLICER blade quad |x|<=half[0] (edge direction), |y|<=half[1]
 *                  (body +y points from the spine to the edge), z = 0 the blade
 *                  normal; thickness; sticky spine circle of spine_radius
 *                  around the segment y = -half[1] (Sec. IV-B)
 *  MPM_SEGMENTS    chain of n_points >= 2 points (body frame) with radius;
 *                  1D contact keeping only the tangential slip (Sec. IV-C)
 *  MPM_ARC         curved needle (Sec. IV-C): the circle of radius half[0]
 *                  about the body origin in the body x-y plane, from angle
 *                  half[1] over half[2] (0 < half[2] <= 2 pi) radians, wire
 *                  radius `radius`; 1D contact along the arc tangent
 *  MPM_MESH_SLICER blade given as an open triangle mesh (Sec. IV-B,
 *                  TriangleMeshSlicer): n_points vertices in points (body
 *                  frame), n_triangles triangles (vertex indices), thickness;
 *                  sticky spine circle of spine_radius around the polyline
 *                  through the n_spine vertices listed in spine (0 or >= 2).
 *                  Normal: the face normal signed by side where the nearest
 *                  point lies inside a triangle, else the nearest-point
 *                  direction.
 * mu_k is the kinetic friction coefficient and c_d the drag factor of Eq. 11.
 * Particles that end a substep inside a sphere or a box are pushed out to its
 * surface (Sec. IV-A); blades, needles and segments push nothing out. */
typedef struct {
    int32_t type;
    int32_t n_points;
    float center[3];
    float quat[4];
    float vel[3];
    float omega[3];
    float mu_k, c_d, margin;
    float radius;
    float half[3];
    float thickness;
    float spine_radius;
    float points[MPM_MAX_SEGMENT_POINTS][3];
    int32_t n_triangles;                           /* MPM_MESH_SLICER */
    int32_t n_spine;                               /* MPM_MESH_SLICER */
    int32_t triangles[MPM_MAX_MESH_TRIANGLES][3];  /* vertex indices into points */
    int32_t spine[MPM_MAX_SPINE_POINTS];           /* vertex indices into points */
} mpm_rigid;

typedef struct mpm_ctx mpm_ctx; /* opaque; owned by the library */

/* ---- lifecycle ------------------------------------------------------- */

/* Create a context on the current CUDA device: the scene container of the
 * paper's object model (Sec. V-A, V-B: a Scene created by the SimulationFactory,
 * here holding n_scenes independent scenes).  `cuda_stream` is a cudaStream_t
 * on which all of the context's work is ordered (NULL: the context creates and
 * owns a non-blocking stream, since substeps are replayed from CUDA graphs,
 * which cannot be captured on the legacy default stream).  Allocates every device buffer the substep needs for
 * cfg->max_particles particles and the scenes' grids up front.
 * Errors: INVALID_ARGUMENT (cfg values), OUT_OF_MEMORY, CUDA. */
int mpm_create(const mpm_config* cfg, void* cuda_stream, mpm_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
int mpm_destroy(mpm_ctx* ctx);

/* Human-readable text of a status code (static storage). */
const char* mpm_status_string(int status);

/* Set a tuning/launch option (MPM_OPT_*).  INVALID_ARGUMENT for an unknown
 * option or an unsupported value. */
int mpm_set_option(mpm_ctx* ctx, int option, int64_t value);

/* Current value of a tuning/launch option (MPM_OPT_*), e.g. what mpm_autotune
 * chose, into *value.  INVALID_ARGUMENT for an unknown option or NULL. */
int mpm_get_option(mpm_ctx* ctx, int option, int64_t* value);

/* ---- factory (Sec. V-B) ---------------------------------------------- */

/* Append n particles to `scene` (a ParticleObject of the paper's object
 * model).  x: (n,3) positions; v: (n,3) initial velocities or NULL (zero);
 * E, nu: (n) per-particle Young's modulus and Poisson ratio, or NULL to use
 * E0, nu0 for all; rho, V0: density and initial particle volume (mass
 * rho*V0), which must equal those of earlier particles of the same scene.
 * C starts at 0 and F at I.  Particle ids within the scene are assigned in
 * call order starting at the scene's current count; *first_id_out (may be
 * NULL) receives the first.  Enqueued on the stream; input buffers may be
 * reused when the call returns.
 * Errors: INVALID_ARGUMENT, CAPACITY, CUDA. */
int mpm_add_particles(mpm_ctx* ctx, int scene, int64_t n, const float* x, const float* v,
                      const float* E, const float* nu, float E0, float nu0, float rho, float V0,
                      int mem, int64_t* first_id_out);

/* Create or replace rigid `rigid_id` (0..MPM_MAX_RIGIDS-1) of `scene`; a type
 * of MPM_RIGID_NONE removes it.  Rigids act on the grid in id order.  The
 * pose given is the pose at the current simulation time; the rigid's
 * accumulated impulse is kept.  Errors: INVALID_ARGUMENT, CUDA. */
int mpm_set_rigid(mpm_ctx* ctx, int scene, int rigid_id, const mpm_rigid* r);

/* ---- simulation ------------------------------------------------------ */

/* Enqueue n_substeps substeps of size dt (seconds) for every scene and
 * return without waiting (the paper's Scene::advance).  Each substep is:
 * sort particles by 4^3-cell brick, P2G, grid update with contact and walls,
 * G2P with the F update (and plasticity).  Errors: INVALID_ARGUMENT, CUDA
 * (launch failures); device-side errors surface in mpm_read_state. */
int mpm_substep(mpm_ctx* ctx, float dt, int n_substeps);

/* Wait (bounded by timeout_ms) for all enqueued work, then copy the
 * requested fields of `scene`'s particles, in particle-id order, into dst[k]
 * (one buffer per set bit of `fields`, in increasing bit order).  This is the
 * paper's blocking Scene::fetchResults.  Returns the scene's sticky device
 * error as an MPM_ERR_* code if one is set (the data is still copied).
 * Host buffers that are page-locked and mapped (cudaHostAlloc, pinned torch
 * tensors) receive X, V, C, F from one kernel writing them over the host link;
 * other host memory is filled through a device staging buffer.
 * Errors: INVALID_ARGUMENT, TIMEOUT, CUDA, OUT_OF_DOMAIN, NONFINITE, INVERTED. */
int mpm_read_state(mpm_ctx* ctx, int scene, uint32_t fields, void* const* dst, int mem);

/* Overwrite fields X, V, C, F of `scene`'s particles from src[k] (id order,
 * one buffer per set bit, increasing bit order); the checkpoint-restore
 * counterpart of mpm_read_state.  Device sources: enqueued.  Host sources:
 * the call returns (bounded wait) once they have been read, so the caller may
 * reuse them; page-locked, mapped ones are read by one kernel over the host
 * link, other host memory through a device staging buffer.
 * Errors: INVALID_ARGUMENT, TIMEOUT, CUDA. */
int mpm_write_state(mpm_ctx* ctx, int scene, uint32_t fields, const void* const* src, int mem);

/* Wait (bounded) and copy the node velocity and mass after the last grid
 * update of `scene`: dst = float (n^3, 4) = (vx, vy, vz, m) per node, node
 * (i,j,k) at (i*n + j)*n + k; nodes untouched by the last P2G read as 0.
 * Errors: INVALID_ARGUMENT, TIMEOUT, CUDA. */
int mpm_read_grid(mpm_ctx* ctx, int scene, float* dst, int mem);

/* Wait (bounded) and return the scene's sticky device error bits
 * (MPM_EBIT_*) in *bits.  Errors: INVALID_ARGUMENT, TIMEOUT, CUDA. */
int mpm_get_error(mpm_ctx* ctx, int scene, uint32_t* bits);

/* Number of particles of a scene (host-side count, no wait). */
int mpm_scene_count(mpm_ctx* ctx, int scene, int64_t* count);

/* Measurement hook (no counterpart in the paper).  Waits (bounded) for the
 * stream, then reports, for the substeps run since the last reset with
 * MPM_OPT_PHASE_TIMING on, the summed device time in milliseconds of each
 * phase: ms[0] sort (scan + scatter), ms[1] P2G (zero for fused substeps that
 * reuse the previous substep's scatter), ms[2] grid update and the reset of
 * the P2G accumulator, ms[3] G2P or the fused G2P + P2G;
 * *n_substeps the number of substeps timed; active[0] / active[1] the numbers
 * of active particle bricks / node bricks of the last substep (all scenes of
 * the last launch group).  reset != 0 clears the sums after reading.
 * Any output pointer may be NULL.  Errors: INVALID_ARGUMENT, TIMEOUT, CUDA. */
int mpm_phase_stats(mpm_ctx* ctx, double* ms, int64_t* n_substeps, int64_t* active, int reset);

/* ---- differentiation ------------------------------------------------- */

/* Start recording a tape at the current state: the state is checkpointed and
 * every following mpm_substep call is recorded (up to tape_max_substeps, with
 * a checkpoint every tape_checkpoint_every substeps).  Requires a context
 * created with tape_checkpoint_every > 0.  Recording runs without graphs.
 * Errors: INVALID_ARGUMENT, STATE, CUDA. */
int mpm_tape_begin(mpm_ctx* ctx);

/* Reverse-mode gradient of a scalar loss L of the final state through every
 * substep recorded since mpm_tape_begin (hand-written adjoint kernels of G2P,
 * grid update and P2G, including the stress and polar/SVD derivatives;
 * segments are recomputed from their checkpoints).  Inputs dL_dx, dL_dv:
 * float (N,3) over ALL particles of the context in scene-major, id order
 * (NULL = zero).  Outputs (same order, may be NULL): dL_dE, dL_dnu (N) for
 * the per-particle Young's modulus and Poisson ratio, dL_dv0 (N,3) for the
 * initial velocities at mpm_tape_begin.  Rigids and walls in contact are
 * differentiated as the masks they apply (the contact law's friction branch
 * is not differentiated: backward returns STATE if any scene has a rigid).
 * Blocks until done (bounded).  Errors: INVALID_ARGUMENT, STATE, TIMEOUT, CUDA. */
int mpm_backward(mpm_ctx* ctx, const float* dL_dx, const float* dL_dv, float* dL_dE,
                 float* dL_dnu, float* dL_dv0, int mem);

/* Reverse-mode gradient with respect to the whole particle state at
 * mpm_tape_begin, for losses of any field of the final state (the same
 * hand-written adjoint kernels and tape as mpm_backward).  bar_in[0..3]: the
 * adjoints dL/dx (N,3), dL/dv (N,3), dL/dC (N,3,3), dL/dF (N,3,3) of the final
 * state over ALL particles of the context, scene-major id order; a NULL array
 * or a NULL entry is zero.  bar_out[0..3] (NULL array or entries = not wanted):
 * dL/dx0, dL/dv0, dL/dC0, dL/dF0 of the state at mpm_tape_begin, same layout;
 * dL_dmu, dL_dlam (N, may be NULL): gradients with respect to the per-particle
 * Lame parameters.  The sort is piecewise constant in x and contributes no
 * derivative; the rest follows mpm_backward (no rigid in any scene, no
 * plasticity).  Blocks until done (bounded).
 * Errors: INVALID_ARGUMENT, STATE, TIMEOUT, CUDA. */
int mpm_backward_state(mpm_ctx* ctx, const float* const* bar_in, float* const* bar_out, float* dL_dmu,
                       float* dL_dlam, int mem);

/* ---- batching -------------------------------------------------------- */

/* Time candidate launch shapes (P2G chunk, threads per CTA and register
 * budget of G2P, persistent CTAs per SM) on `trial_substeps` substeps of size dt and keep the fastest.
 * Each trial is timed as the user's substeps run: one graph replay of the
 * substeps (rounded up to an even count) when graphs are on, else direct
 * launches.  The particle state, keys, clocks and impulses are restored afterwards, so
 * the simulation does not advance.  *best_ms_out (may be NULL) receives the
 * best time per substep.  Blocks.  Errors: INVALID_ARGUMENT, CUDA, TIMEOUT. */
int mpm_autotune(mpm_ctx* ctx, float dt, int trial_substeps, float* best_ms_out);

/* ---- allocation-free brick sort --------------------------------------- */

#define MPM_NOALLOC_MAX_PARTICLES 1048576 /* largest N accepted                  */
#define MPM_NOALLOC_MAX_GRID 256          /* largest n (nodes per dimension)     */

/* The particle sort of mpm_substep (ordering by the 4^3-node brick that holds
 * each particle's base cell) for callers that must not allocate device memory
 * while they run: a host loop that cannot take the device-wide synchronisation
 * of cudaMalloc/cudaFree every frame, work recorded into CUDA graphs (where
 * allocation is not allowed), or integrations that only lend the library the
 * buffers they own.  The paper has no counterpart to this call.
 *
 * x: device float (N,3) positions of one grid of n^3 nodes (dx = 1/n);
 * perm: device int[N], receives the particle indices ordered by brick (the
 * order inside a brick is unspecified); brick_start: device int[(n/4)^3 + 1]
 * or NULL, receives the first sorted slot of each brick and N at the end.
 * Work is enqueued on `cuda_stream` (a cudaStream_t; NULL = legacy stream).
 *
 * It allocates nothing: its scratch is one static device array of
 * 10,486,784 bytes that every device loading the library reserves until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current, and looks it up
 * again after that device's context was reset and recreated; make that first
 * call (and the first after a reset) before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU race and must be serialised by the caller.
 * Errors: INVALID_ARGUMENT (n not a multiple of 4 or < 8, N < 0, NULL
 * buffers), CAPACITY (N > MPM_NOALLOC_MAX_PARTICLES or n > MPM_NOALLOC_MAX_GRID),
 * CUDA (launch or symbol lookup failed). */
int mpm_sort_bricks_noalloc(int n, int64_t N, const float* x, int* perm, int* brick_start, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPM_GB300_H */
