// Brick sort that allocates nothing: the counting sort of particles by the
// 4^3-node brick of their base cell, run entirely in a fixed scratch area
// that the library reserves statically on every device it is loaded on.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. a per-frame loop of a host application that cannot afford the device
// synchronisation cudaMalloc/cudaFree imply, code that records work into a
// CUDA graph (allocations are not allowed there), or integrations that hand
// the library only the buffers they own.
//
// Scratch: one static __device__ array (below) of 10,486,784 bytes, shared by
// every call on that device and kept until the process exits.  Host code
// only sees a stand-in for its name, so the device address is obtained with
// cudaGetSymbolAddress once per device, on the first call made with that
// device current (and again if that device's context was reset and
// recreated, which the context id tells).  Calls that overlap on the GPU (different streams or host
// threads) use the same scratch and race: serialise them.
#include <mutex>

#include "mpm_device.cuh"

namespace {

constexpr int kNaMaxParticles = 1 << 20;  // MPM_NOALLOC_MAX_PARTICLES
constexpr int kNaMaxGrid = 256;           // MPM_NOALLOC_MAX_GRID
constexpr int kNaMaxBricks = (kNaMaxGrid / 4) * (kNaMaxGrid / 4) * (kNaMaxGrid / 4);
constexpr int kNaScanThreads = 1024;

// keys[N] | ranks[N] | counts[bricks] | offsets[bricks + 1]
constexpr size_t kNaScratchInts = 2 * (size_t)kNaMaxParticles + 2 * (size_t)kNaMaxBricks + 256;
static __device__ __align__(256) int g_scratch[kNaScratchInts];

struct NaScratch {
    int* keys;
    int* ranks;
    int* counts;
    int* offsets;
};

static NaScratch view(int* base)
{
    NaScratch s;
    s.keys = base;
    s.ranks = base + kNaMaxParticles;
    s.counts = base + 2 * (size_t)kNaMaxParticles;
    s.offsets = base + 2 * (size_t)kNaMaxParticles + kNaMaxBricks;
    return s;
}

__global__ void k_na_clear(int* counts, int nbricks)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbricks) counts[i] = 0;
}

// Key (brick of the base cell, decided as floor(fma(x, n, -0.5)), clamped to
// the grid) and rank inside the brick from one atomic per distinct key per warp.
__global__ void k_na_keys(const float* x, int N, int n, NaScratch s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < N;
    int key = 0;
    if (valid) {
        int c0, c1, c2;
        mpm::base_cell(x[3 * (size_t)i], n, c0);
        mpm::base_cell(x[3 * (size_t)i + 1], n, c1);
        mpm::base_cell(x[3 * (size_t)i + 2], n, c2);
        const int nb = n / 4;
        key = ((c0 >> 2) * nb + (c1 >> 2)) * nb + (c2 >> 2);
    }
    const unsigned full = 0xffffffffu;
    const unsigned active = __ballot_sync(full, valid);
    const unsigned peers = __match_any_sync(full, valid ? key : -1) & active;
    if (valid) {
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&s.counts[key], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        s.keys[i] = key;
        s.ranks[i] = base + __popc(peers & ((1u << lane) - 1u));
    }
}

// Exclusive scan of the brick counts by one CTA (no inter-CTA waiting).
__global__ void __launch_bounds__(kNaScanThreads) k_na_scan(NaScratch s, int nbricks, int* brick_start)
{
    __shared__ int warp_sum[kNaScanThreads / 32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nbricks; base += kNaScanThreads) {
        const int i = base + tid;
        const int c = i < nbricks ? s.counts[i] : 0;
        int incl = c;
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = warp_sum[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += t;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        const int excl = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + incl - c;
        if (i < nbricks) {
            s.offsets[i] = excl;
            if (brick_start) brick_start[i] = excl;
        }
        __syncthreads();
        if (tid == kNaScanThreads - 1) carry = excl + c;
        __syncthreads();
    }
    if (tid == 0) {
        s.offsets[nbricks] = carry;
        if (brick_start) brick_start[nbricks] = carry;
    }
}

// Every slot is written exactly once: the ranks and the brick counts come from
// the same atomics, so offsets[key] + rank covers [0, N) without gaps.
__global__ void k_na_scatter(int N, NaScratch s, int* perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int dst = s.offsets[s.keys[i]] + s.ranks[i];
    if (dst >= 0 && dst < N) perm[dst] = i;
}

// Driver calls reached through the runtime (no link against libcuda): the
// current context and its unique id, so that a cached address is never used
// in a context other than the one it was looked up in (a cudaDeviceReset
// destroys the primary context; the next one gets a new id).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

struct ScratchSlot {
    unsigned long long ctx_id = 0;
    int* addr = nullptr;
};

std::mutex g_mu;
ScratchSlot g_slot[64];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_driver_looked_up = false;

// Id of the current context, 0 when the driver entry points are unavailable.
unsigned long long current_context_id()
{
    if (!g_driver_looked_up) {
        g_driver_looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current && g_ctx_id && g_ctx_current(&ctx) == 0 && ctx && g_ctx_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of the scratch array in the current device's context: looked
// up with cudaGetSymbolAddress on the first call with that device (and
// context) current, then reused.
cudaError_t scratch_address(int** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    // make sure the device's context exists before asking for its id
    if (!g_slot[dev].addr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_slot[dev].addr = static_cast<int*>(p);
        g_slot[dev].ctx_id = current_context_id();
    } else {
        const unsigned long long id = current_context_id();
        if (id != g_slot[dev].ctx_id) {  // the context was reset and recreated
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return e;
            g_slot[dev].addr = static_cast<int*>(p);
            g_slot[dev].ctx_id = id;
        }
    }
    *out = g_slot[dev].addr;
    return cudaSuccess;
}

}  // namespace

extern "C" int mpm_sort_bricks_noalloc(int n, int64_t N, const float* x, int* perm, int* brick_start,
                                       void* cuda_stream)
{
    if (n < 8 || n % 4 != 0 || N < 0) return MPM_ERR_INVALID_ARGUMENT;
    if (n > kNaMaxGrid || N > kNaMaxParticles) return MPM_ERR_CAPACITY;  // beyond the static scratch
    if (N > 0 && (!x || !perm)) return MPM_ERR_INVALID_ARGUMENT;
    int* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return MPM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const NaScratch sc = view(base);
    const int nb = n / 4, nbricks = nb * nb * nb;
    k_na_clear<<<(nbricks + 255) / 256, 256, 0, s>>>(sc.counts, nbricks);  // counts start at zero every call
    if (N > 0) k_na_keys<<<(int)((N + 255) / 256), 256, 0, s>>>(x, (int)N, n, sc);
    k_na_scan<<<1, kNaScanThreads, 0, s>>>(sc, nbricks, brick_start);
    if (N > 0) k_na_scatter<<<(int)((N + 255) / 256), 256, 0, s>>>((int)N, sc, perm);
    return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}
