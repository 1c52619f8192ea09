// Forward substep kernels of the MLS-MPM transfer loop (arXiv 2502.18437,
// Algorithm 1) for GB300 (sm_103a):
//   k_scan     brick histogram -> particle offsets, active particle-brick and
//              node-brick lists (tile sums kept by the key producers: no
//              inter-CTA waits, empty tiles skipped)
//   k_scatter  counting-sort scatter: permutation sorted slot -> particle
//   k_p2g      P2G (Eq. 1, Eq. 8): balanced per-cell work items summed in
//              registers into shared-memory 6^3 node windows per brick, flushed
//              to HBM with vector atomics; leaves the permutation in cell order
//   k_grid     grid update (Eq. 3), rigid contact (Sec. IV, Eq. 11, Eq. 12),
//              domain walls (k_grid_plain where no scene has a rigid)
//   k_grid_clear  reset of the P2G accumulator
//   k_g2p      G2P (Eq. 4, Eq. 9, Eq. 10) with the 2x2x2-brick velocity halo
//              staged by bulk-copy TMA, plasticity, next brick key + rank
#include <cstdint>
#include <cstdio>

#include "mpm_transfer.cuh"

namespace mpm {

// ----------------------------------------------------------------- scan
//
// A scan tile is 2^tile_shift consecutive bricks of one scene (tiles never
// straddle scenes).  Each brick contributes (particles, is an active particle
// brick, is an active node brick); a node brick is active when it or one of its
// 7 lower neighbours (-1 in any subset of the axes) holds particles, since a
// particle's 3-node stencil reaches at most 2 nodes beyond its base cell, i.e.
// into the next brick.  The key producers (G2P, k_prepare) count particles per
// brick, flag those node bricks when the first particles enter a brick, and add
// each tile's totals as they go.  So every CTA of the scan (one per tile of
// the range) knows its exclusive prefix from the tile totals before it,
// without waiting for another CTA; a tile with no active node brick has
// nothing to write and returns at once.  The active particle-brick list holds
// the bricks of at least kBigBrick particles first (in brick order), then the
// others: the fourth tile total counts the former, and the grand total of the
// range places the latter.

__device__ __forceinline__ int4 add4(int4 a, int4 b) { return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

__device__ __forceinline__ int4 shfl_up4(int4 v, int d)
{
    return make_int4(__shfl_up_sync(kFull, v.x, d), __shfl_up_sync(kFull, v.y, d), __shfl_up_sync(kFull, v.z, d),
                     __shfl_up_sync(kFull, v.w, d));
}

__global__ void __launch_bounds__(kScanThreads) k_scan(StepArgs a)
{
    __shared__ int4 s_warp[kScanThreads / 32];
    __shared__ int s_wtot[kScanThreads / 32];
    __shared__ int4 s_prefix;
    __shared__ int s_big_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SortBufs& sb = a.sb;
    const int tile = a.r.t0 + blockIdx.x;
    const bool last = blockIdx.x == a.r.nt - 1;
    if (blockIdx.x == 0 && tid == 0) {
        sb.counters[CTR_WORK_P2G] = 0;
        sb.counters[CTR_WORK_GRID] = 0;
        sb.counters[CTR_WORK_G2P] = 0;
    }
    const int4 own = __ldcg(&sb.tile_sum[tile]);
    if (own.z == 0 && !last) return;  // no active node brick (hence no particle) here

    // exclusive prefix: the totals of the range's tiles before this one; and the
    // range's count of big bricks (the start of the small bricks in the list)
    int4 pre = make_int4(0, 0, 0, 0);
    int wtot = 0;
    for (int t = a.r.t0 + tid; t < a.r.t0 + a.r.nt; t += kScanThreads) {
        const int4 ts = __ldcg(&sb.tile_sum[t]);
        if (t < tile) pre = add4(pre, ts);
        wtot += ts.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pre.x += __shfl_xor_sync(kFull, pre.x, o);
        pre.y += __shfl_xor_sync(kFull, pre.y, o);
        pre.z += __shfl_xor_sync(kFull, pre.z, o);
        pre.w += __shfl_xor_sync(kFull, pre.w, o);
        wtot += __shfl_xor_sync(kFull, wtot, o);
    }
    if (lane == 0) {
        s_warp[warp] = pre;
        s_wtot[warp] = wtot;
    }
    __syncthreads();
    if (tid == 0) {
        int4 p = make_int4(0, 0, 0, 0);
        int wt = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) {
            p = add4(p, s_warp[w]);
            wt += s_wtot[w];
        }
        s_prefix = p;
        s_big_total = wt;
        if (last) {
            const int4 tot = add4(p, own);
            if (tot.x == a.r.np) {
                sb.counters[CTR_N_ACT] = tot.y;
                sb.counters[CTR_N_NACT] = tot.z;
            } else {
                // histogram and particle count disagree: skip this substep's work
                sb.counters[CTR_N_ACT] = 0;
                sb.counters[CTR_N_NACT] = 0;
                atomicOr(&a.err[a.r.s0], MPM_EBIT_INTERNAL);
            }
        }
    }
    __syncthreads();
    if (own.z == 0) return;
    int4 run = s_prefix;
    const int big_total = s_big_total;

    // scene of the tile
    int s;
    {
        int lo = a.r.s0, hi = a.r.s1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.scenes[mid].tile_base <= tile) lo = mid;
            else hi = mid - 1;
        }
        s = lo;
    }
    const SceneDev& sc = a.scenes[s];
    const int tb = 1 << sb.tile_shift;
    const int b0 = sc.brick_base + (tile - sc.tile_base) * tb;
    const int b1 = min(b0 + tb, sc.brick_base + sc.nb * sc.nb * sc.nb);
    for (int chunk = b0; chunk < b1; chunk += kScanChunk) {
        const int first = chunk + tid * kScanItems;
        int c[kScanItems];
        unsigned pf = 0, nf = 0, bf = 0;
        int4 local = make_int4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int b = first + k;
            c[k] = 0;
            if (b < b1) {
                c[k] = __ldcg(&sb.cnt[b]);
                const int flag = __ldcg(&sb.nflag[b]);  // reset by k_grid_clear
                if (c[k] > 0) pf |= 1u << k;
                if (c[k] >= kBigBrick) bf |= 1u << k;
                if (flag) nf |= 1u << k;  // a non-empty brick always flags itself
                local.x += c[k];
            }
        }
        local.y = __popc(pf);
        local.z = __popc(nf);
        local.w = __popc(bf);
        // block exclusive scan of (particles, pbricks, nbricks)
        int4 incl = local;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int4 t = shfl_up4(incl, d);
            if (lane >= d) incl = add4(incl, t);
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int4 w = lane < kScanThreads / 32 ? s_warp[lane] : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int4 t = shfl_up4(w, d);
                if (lane >= d) w = add4(w, t);
            }
            if (lane < kScanThreads / 32) s_warp[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int4 excl = make_int4(incl.x - local.x, incl.y - local.y, incl.z - local.z, incl.w - local.w);
        if (warp > 0) excl = add4(excl, s_warp[warp - 1]);
        excl = add4(excl, run);
        // list positions: big bricks from excl.w, the others after all big bricks
        int po = a.r.p0 + excl.x, bi = excl.w, si = big_total + excl.y - excl.w, ni = excl.z;
        if (excl.y + local.y > a.r.nbr || ni + local.z > a.r.nbr || bi + local.w > big_total ||
            si + local.y - local.w > a.r.nbr) {  // tile sums out of step with the bricks
            atomicOr(&a.err[a.r.s0], MPM_EBIT_INTERNAL);
            pf = nf = 0u;
        }
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int b = first + k;
            if (pf & (1u << k)) {
                const int pi = (bf & (1u << k)) ? bi++ : si++;
                sb.off[b] = po;
                sb.act_brick[pi] = b;
                sb.act_start[pi] = po;
                sb.act_count[pi] = c[k];
                sb.act_scene[pi] = s;
            }
            if (nf & (1u << k)) {
                sb.nact_brick[ni] = b;
                sb.nact_scene[ni] = s;
                ++ni;
            }
            po += c[k];
        }
        run = add4(run, s_warp[kScanThreads / 32 - 1]);
        __syncthreads();  // s_warp is rewritten by the next chunk
    }
}

// Counting-sort scatter; also clears the range's tile sums for the next
// substep (the scan has read them).  write_perm = 0 only clears (the adjoint
// reuses a recorded permutation).
// Each thread takes kScatterPer particles, 256 apart, with their loads issued
// together (a 1M-particle range in one wave of CTAs).
__global__ void __launch_bounds__(256) k_scatter(StepArgs a, int write_perm)
{
    const int g0 = blockIdx.x * (256 * kScatterPer) + threadIdx.x;
    int key[kScatterPer], rank[kScatterPer], dst[kScatterPer];
#pragma unroll
    for (int u = 0; u < kScatterPer; ++u) {
        const int g = g0 + u * 256;
        key[u] = -1;
        rank[u] = 0;
        if (write_perm && g < a.r.np) {
            key[u] = a.sb.key[a.r.p0 + g];
            rank[u] = a.sb.rank[a.r.p0 + g];
        }
    }
#pragma unroll
    for (int u = 0; u < kScatterPer; ++u) {
        const int brick = key[u] >> 6;
        dst[u] = (key[u] >= 0 && brick >= a.r.bb0 && brick < a.r.bb0 + a.r.nbr) ? __ldg(&a.sb.off[brick]) + rank[u] : -1;
    }
#pragma unroll
    for (int u = 0; u < kScatterPer; ++u) {
        const int g = g0 + u * 256;
        if (write_perm && g < a.r.np) {
            if (dst[u] >= a.r.p0 && dst[u] < a.r.p0 + a.r.np) {
                a.sb.perm[dst[u]] = a.r.p0 + g;
                a.sb.scell[dst[u]] = (unsigned char)(key[u] & 63);
            } else {
                atomicOr(&a.err[a.r.s0], MPM_EBIT_INTERNAL);
            }
        }
        if (g < a.r.nt) a.sb.tile_sum[a.r.t0 + g] = make_int4(0, 0, 0, 0);
    }
}

// Keys and ranks of the stored particles after the host changed positions
// (new particles, state writes).  Stored particles may be in any order here, so
// the tiles' particle counts are first summed per block in shared memory (with
// at most kPrepTiles tiles in the range; else each warp adds its own).
constexpr int kPrepTiles = 2048;

__global__ void __launch_bounds__(256) k_prepare(StepArgs a, PState st)
{
    __shared__ int s_tile[kPrepTiles];
    const bool block_sums = a.r.nt <= kPrepTiles;
    if (block_sums)
        for (int t = threadIdx.x; t < a.r.nt; t += blockDim.x) s_tile[t] = 0;
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = a.r.p0 + g;
    const bool valid = g < a.r.np;
    int key = 0, scene = a.r.s0;
    unsigned ebits = 0;
    if (valid) {
        int lo = a.r.s0, hi = a.r.s1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.scenes[mid].p_begin <= i) lo = mid;
            else hi = mid - 1;
        }
        scene = lo;
    }
    const SceneDev sc = a.scenes[scene];
    if (valid) {
        unsigned ood = 0;
        key = cell_key(sc, st.x[i], st.x[a.cap + i], st.x[2 * a.cap + i], ood);
        if (ood) ebits |= MPM_EBIT_OUT_OF_DOMAIN;
    }
    const int rank = aggregated_rank_mark(a.sb, sc, key >> 6, valid, !block_sums);
    if (valid) {
        a.sb.key[i] = key;
        a.sb.rank[i] = rank;
        if (ebits) atomicOr(&a.err[scene], ebits);
        if (block_sums)
            atomicAdd(&s_tile[sc.tile_base + (((key >> 6) - sc.brick_base) >> a.sb.tile_shift) - a.r.t0], 1);
    }
    if (block_sums) {
        __syncthreads();
        for (int t = threadIdx.x; t < a.r.nt; t += blockDim.x)
            if (s_tile[t]) atomicAdd(&a.sb.tile_sum[a.r.t0 + t].x, s_tile[t]);
    }
}

// ------------------------------------------------------------------ P2G
//
// One CTA per active particle brick (4^3 cells, a 6^3-node window), 192
// threads.  Per pass over up to PER x 192 particles of the brick:
//   A1. one thread per particle: base cell (stored by the sort beside the
//      permutation) and rank inside the cell;
//   (warp 0) the cells' particles are cut into at most 64 balanced work items
//      (build_items), so that the lanes of a warp run loops of nearly equal
//      length instead of as long as the warp's fullest cell;
//   A2. stress, weights and P2G coefficients into a record in shared memory at
//      slot base(warp) + (position in item) x 33 + lane of the item, so that
//      the 32 lanes of a warp read 32 consecutive words in phase B and the
//      particles of one item (consecutive lanes here when the input is in cell
//      order) write to different banks; a pass whose two item warps need more
//      than the pass's record slots falls back to cell-sorted slots.  The pass's slots
//      of the permutation are rewritten in cell order (cell_order), so that G2P
//      gathers a warp's 27-node stencils from a few neighbouring cells;
//   B.  thread (item, slice i) sums, in registers, the contributions of its
//      item's particles to the 9 nodes cell + (i, j, k) and stages the sums;
//   C.  thread (cell, slice i) adds the staged sums of its cell's items and
//      adds them to slice i's copy of the 6^3 window: the 64 cells of a slice
//      never write the same node at once, so no atomics are needed.
// At the end of the pass the window is added to HBM with one vector reduction
// per node.  Stage and windows reuse the record slots.

__device__ __forceinline__ void prefetch_l2(const float* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

constexpr int kP2GSlotPitch = 33;  // 32 lanes + 1: rows of one item fall in different banks
// record slots of a pass of PER x 192 particles (the rows of the interleaved
// layout; 768-particle passes need 24).  A smaller record area leaves more of
// the SM's shared storage to L1.
template <int PER>
struct P2GShape {
    static constexpr int slots = (PER == 4 ? 24 : 21) * kP2GSlotPitch;
};
constexpr int kSliceNodes = 4 * 36;  // node planes x = slice .. slice + 3 of the 6^3 window
constexpr int kStageFloats = 36 * 3 * 64;  // (9 nodes x 4 values) x 3 slices x 64 items
constexpr int kWinFloats = 3 * 4 * kSliceNodes;  // the slices' windows, after the stage

// MODE: kP2GStress (MLS-MPM: the Kirchhoff stress, stored by G2P or computed
// from F) or kP2GConstraint (PB-MPM: the co-rotational constraint replaces C
// and there is no stress term).
enum { kP2GStress = 0, kP2GConstraint = 1 };

template <int PER, int MODE>
__global__ void __launch_bounds__(kP2GThreads, 4) k_p2g(StepArgs a)
{
    constexpr int CHUNK = PER * kP2GThreads;
    constexpr int kP2GSlots = P2GShape<PER>::slots;
    static_assert(CHUNK <= kP2GSlots, "a pass fits the record slots");
    static_assert(kStageFloats + kWinFloats <= kItemRecFields * kP2GSlots, "stage and windows reuse the record slots");
    extern __shared__ __align__(16) float rec_dyn[];
    float(*rec)[kP2GSlots] = reinterpret_cast<float(*)[kP2GSlots]>(rec_dyn);  // [kItemRecFields][kP2GSlots]
    // written once phase B has read every record: the staged item sums [36][3][64]
    // and one window per slice (slice i writes node planes x = i..i+3 only, so the
    // slices' writes never collide), added to HBM at the end of each pass
    float* stage = rec_dyn;
    float(*win)[4][kSliceNodes] = reinterpret_cast<float(*)[4][kSliceNodes]>(rec_dyn + kStageFloats);
    __shared__ int cell_cnt[64], cell_off[65];
    __shared__ short it_cell[64], it_beg[64], it_len[64], c_full[64], c_nf[64], c_rem[64];
    __shared__ int s_item, s_nitems, s_len[3];
    const int tid = threadIdx.x;
    const int t = tid & 63, slice = tid >> 6;
    const int n_act = a.sb.counters[CTR_N_ACT];
    const int cap = a.cap;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.sb.counters[CTR_WORK_P2G], 1);
        if (tid < 64) cell_cnt[tid] = 0;
        __syncthreads();
        const int item = s_item;
        if (item >= n_act) break;
        const int b = a.sb.act_brick[item], start = a.sb.act_start[item], count = a.sb.act_count[item];
        const int scene = a.sb.act_scene[item];
        const SceneDev sc = a.scenes[scene];
        const int n = sc.n, nb = sc.nb, lb = b - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float fn = (float)n, dxs = 1.0f / fn;
        const float m = sc.m_p;
        const float kA = a.dt * sc.V0 * 4.0f * fn * fn;
        unsigned ebits = 0;

        for (int c0 = 0; c0 < count; c0 += CHUNK) {
            const int cn = min(CHUNK, count - c0);
            // A1: cell and rank of each particle of the pass
            int pp[PER], pc[PER], pr[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int k = tid + u * kP2GThreads;
                pc[u] = -1;
                if (k < cn) {
                    const int p = a.sb.perm[start + c0 + k];
                    pp[u] = p;
                    if (a.cell_order) {
                        // the sort stored each slot's cell: no dependent load of x here
                        pc[u] = a.sb.scell[start + c0 + k];
                    } else {
                        // a recorded permutation (differentiation): the cell from x
                        int c[3];
                        const unsigned ood = base_cell(a.in.x[p], n, c[0]) | base_cell(a.in.x[cap + p], n, c[1]) |
                                             base_cell(a.in.x[2 * cap + p], n, c[2]);
                        if (ood) ebits |= MPM_EBIT_OUT_OF_DOMAIN;
                        const int l0 = min(max(c[0] - ox, 0), 3), l1 = min(max(c[1] - oy, 0), 3),
                                  l2 = min(max(c[2] - oz, 0), 3);
                        pc[u] = (l0 * 4 + l1) * 4 + l2;
                    }
                    pr[u] = atomicAdd(&cell_cnt[pc[u]], 1);
                }
            }
            // the pass's particle fields start towards L2 while warp 0 builds the items
            // (phase A2 then loads them from L2 rather than from HBM)
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (pc[u] < 0) continue;
                const int p = pp[u];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    prefetch_l2(a.in.x + (size_t)q * cap + p);
                    prefetch_l2(a.in.v + (size_t)q * cap + p);
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) prefetch_l2(a.in.C + (size_t)q * cap + p);
                if (MODE == kP2GStress && a.tau_valid) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) prefetch_l2(a.in.tau + (size_t)q * cap + p);
                } else {
#pragma unroll
                    for (int q = 0; q < 9; ++q) prefetch_l2(a.in.F + (size_t)q * cap + p);
                }
            }
            __syncthreads();
            if (tid < 32)
                build_items(cell_cnt, cell_off, cn, it_cell, it_beg, it_len, &s_nitems, c_full, c_nf, c_rem, s_len);
            __syncthreads();
            const int L = s_len[0], n_items = s_nitems;
            const int rows0 = s_len[1], rows1 = s_len[2];  // record rows of the two item warps
            const bool inter = kP2GSlotPitch * (rows0 + rows1) <= kP2GSlots;
            const float invL = 1.0f / (float)L;
            if (tid < 64) cell_cnt[tid] = 0;  // counts of the next pass (last read before the barrier)
            // A2: records at their slots
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (pc[u] < 0) continue;
                const int c = pc[u], r = pr[u], nf = c_nf[c];
                // the pass's slots in cell order: G2P then reads (and stores) the
                // particles of a warp from a few neighbouring cells
                if (a.cell_order) a.sb.perm[start + c0 + cell_off[c] + r] = pp[u];
                int slot;
                if (!inter) {
                    slot = cell_off[c] + r;
                } else {
                    int ti, it;
                    if (r < nf * L) {
                        const int j = div_small(r, invL);
                        ti = c_full[c] + j;
                        it = r - j * L;
                    } else {
                        ti = c_rem[c];
                        it = r - nf * L;
                    }
                    slot = (ti < 32 ? 0 : kP2GSlotPitch * rows0) + it * kP2GSlotPitch + (ti & 31);
                }
                const int p = pp[u];
                int bc[3];
                float f[3], w[9];
                ebits |= particle_weights(a.in.x[p], a.in.x[cap + p], a.in.x[2 * cap + p], n, bc, f, w);
                float C[9], v[3], t6[6];
#pragma unroll
                for (int q = 0; q < 9; ++q) C[q] = a.in.C[(size_t)q * cap + p];
#pragma unroll
                for (int q = 0; q < 3; ++q) v[q] = a.in.v[(size_t)q * cap + p];
                if (MODE == kP2GConstraint) {
                    float F[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) F[q] = a.in.F[(size_t)q * cap + p];
                    pb_constraint(F, a.dt, a.pb_beta, C);
#pragma unroll
                    for (int q = 0; q < 6; ++q) t6[q] = 0.f;
                } else if (a.tau_valid) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) t6[q] = a.in.tau[(size_t)q * cap + p];
                } else {
                    // stress of the current F (after host writes, or seeding a fused run)
                    float F[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) F[q] = a.in.F[(size_t)q * cap + p];
                    const float mu = sc.pp_mat ? a.in.mu[p] : sc.mu, lam = sc.pp_mat ? a.in.lam[p] : sc.lam;
                    ebits |= constitutive(a.model, 0, 0.f, mu, lam, F, t6);
                }
                float q3[3], Ad[9];
                p2g_coeffs(m, kA, dxs, v, C, t6, f, q3, Ad);
                put_item_record<kP2GSlots>(rec, slot, f, q3, Ad);
            }
            __syncthreads();
            // B: item sums in registers, then staged
            float2 acc_a[9], acc_b[9];  // (p_x, p_y), (p_z, weight)
#pragma unroll
            for (int q = 0; q < 9; ++q) acc_a[q] = acc_b[q] = make_float2(0.f, 0.f);
            if (t < n_items)
                item_accumulate<kP2GSlots>(rec, inter ? (t < 32 ? 0 : kP2GSlotPitch * rows0) + (t & 31) : it_beg[t],
                                           inter ? kP2GSlotPitch : 1,
                                           it_len[t], slice, acc_a, acc_b);
            __syncthreads();
            for (int q = tid; q < kWinFloats; q += kP2GThreads) (&win[0][0][0])[q] = 0.0f;
            if (t < n_items) {
                float* st = stage + slice * 64 + t;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    st[(4 * q) * 192] = acc_b[q].y * m;
                    st[(4 * q + 1) * 192] = acc_a[q].x;
                    st[(4 * q + 2) * 192] = acc_a[q].y;
                    st[(4 * q + 3) * 192] = acc_b[q].x;
                }
            }
            __syncthreads();
            // C: cell owners add their items' sums to their slice's window
            {
                const int c = t, nf = c_nf[c], f0 = c_full[c], pr_item = c_rem[c];
                const int cx = c >> 4, cy = (c >> 2) & 3, cz = c & 3;
                float sum[36];
#pragma unroll
                for (int q = 0; q < 36; ++q) sum[q] = 0.f;
                const bool any = nf > 0 || pr_item >= 0;
                for (int j = 0; j <= nf; ++j) {
                    const int it = j < nf ? f0 + j : pr_item;
                    if (it < 0) break;
                    const float* st = stage + slice * 64 + it;
#pragma unroll
                    for (int q = 0; q < 36; ++q) sum[q] += st[q * 192];
                }
                // for one (j, k) the 64 cells of a slice write distinct nodes (the two
                // warps of a slice cover disjoint x ranges); a node written for (j, k)
                // is read for another (j, k) by a neighbour lane: warp barrier between
                float(*w)[kSliceNodes] = win[slice];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    if (any) {
                        const int node = cx * 36 + (cy + q / 3) * 6 + (cz + q % 3);
                        w[0][node] += sum[4 * q];
                        w[1][node] += sum[4 * q + 1];
                        w[2][node] += sum[4 * q + 2];
                        w[3][node] += sum[4 * q + 3];
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            // the pass's window to HBM, one vector reduction per node (read before
            // the next pass's records overwrite it: two barriers away)
            for (int q = tid; q < kWinNodes; q += kP2GThreads) {
                const int X = q / 36, yz = q % 36;
                float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int sl = 0; sl < 3; ++sl) {
                    const int cx = X - sl;
                    if (cx < 0 || cx > 3) continue;
#pragma unroll
                    for (int comp = 0; comp < 4; ++comp) s4[comp] += win[sl][comp][cx * 36 + yz];
                }
                if (s4[0] == 0.0f) continue;
                const int gi = ox + X, gj = oy + yz / 6, gk = oz + yz % 6;
                if (gi >= n || gj >= n || gk >= n) continue;
                red_add_v4(&a.G[node_index(sc, gi, gj, gk)], s4[0], s4[1], s4[2], s4[3]);
            }
        }
        if (ebits) atomicOr(&a.err[scene], ebits);
        __syncthreads();
    }
}

// ----------------------------------------------------------- grid update


// Nearest point q of segment [a, b] to p (endpoint projections keep the
// segment); returns |p - q|.
__device__ __forceinline__ float closest_on_segment_f(float p0, float p1, float p2, const float* a, const float* b,
                                                      float q[3])
{
    const float e0 = b[0] - a[0], e1 = b[1] - a[1], e2 = b[2] - a[2];
    const float L2 = e0 * e0 + e1 * e1 + e2 * e2;
    float u = L2 > 0.f ? ((p0 - a[0]) * e0 + (p1 - a[1]) * e1 + (p2 - a[2]) * e2) / L2 : 0.f;
    u = fminf(fmaxf(u, 0.f), 1.f);
    q[0] = a[0] + u * e0;
    q[1] = a[1] + u * e1;
    q[2] = a[2] + u * e2;
    const float d0 = p0 - q[0], d1 = p1 - q[1], d2 = p2 - q[2];
    return sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
}

// Nearest point q of triangle (a, b, c) to p: the orthogonal projection when
// its barycentric coordinates (2x2 normal equations of the plane) lie inside
// (inside = true), else the nearest of the three edges' nearest points.
__device__ __forceinline__ float closest_on_triangle_f(float p0, float p1, float p2, const float* a, const float* b,
                                                       const float* c, float q[3], bool& inside)
{
    const float e0[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e1[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const float ap[3] = {p0 - a[0], p1 - a[1], p2 - a[2]};
    const float d00 = e0[0] * e0[0] + e0[1] * e0[1] + e0[2] * e0[2];
    const float d01 = e0[0] * e1[0] + e0[1] * e1[1] + e0[2] * e1[2];
    const float d11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const float d20 = ap[0] * e0[0] + ap[1] * e0[1] + ap[2] * e0[2];
    const float d21 = ap[0] * e1[0] + ap[1] * e1[1] + ap[2] * e1[2];
    const float den = d00 * d11 - d01 * d01;
    inside = false;
    if (den > 0.f) {
        const float s = (d11 * d20 - d01 * d21) / den, t = (d00 * d21 - d01 * d20) / den;
        if (s >= 0.f && t >= 0.f && s + t <= 1.f) {
#pragma unroll
            for (int i = 0; i < 3; ++i) q[i] = a[i] + s * e0[i] + t * e1[i];
            inside = true;
            const float d0 = p0 - q[0], d1 = p1 - q[1], d2 = p2 - q[2];
            return sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        }
    }
    float qa[3], qb[3], qc[3];
    const float da = closest_on_segment_f(p0, p1, p2, a, b, qa), db = closest_on_segment_f(p0, p1, p2, b, c, qb),
                dc = closest_on_segment_f(p0, p1, p2, c, a, qc);
    float best = da;
    q[0] = qa[0]; q[1] = qa[1]; q[2] = qa[2];
    if (db < best) { best = db; q[0] = qb[0]; q[1] = qb[1]; q[2] = qb[2]; }
    if (dc < best) { best = dc; q[0] = qc[0]; q[1] = qc[1]; q[2] = qc[2]; }
    return best;
}

// Region of the triangle-mesh slicer at body point p (3 sticky spine, 1
// regular, 0 none) and its body-frame normal nl.
__device__ __forceinline__ int mesh_slicer_region(const RigidCur& R, float p0, float p1, float p2, float nl[3])
{
    float dsp = 3.4e38f;
    for (int k = 0; k + 1 < R.n_spine; ++k) {
        const float* a = R.shape.pts + 3 * R.shape.spine[k];
        const float* b = R.shape.pts + 3 * R.shape.spine[k + 1];
        float q[3];
        dsp = fminf(dsp, closest_on_segment_f(p0, p1, p2, a, b, q));
    }
    if (dsp < R.spine_radius + R.margin) return 3;
    float best = 3.4e38f, bq[3] = {0.f, 0.f, 0.f};
    int bt = -1;
    bool binside = false;
    for (int k = 0; k < R.n_tris; ++k) {
        const unsigned char* tv = R.shape.tris + 3 * k;
        float q[3];
        bool inside;
        const float l = closest_on_triangle_f(p0, p1, p2, R.shape.pts + 3 * tv[0], R.shape.pts + 3 * tv[1],
                                              R.shape.pts + 3 * tv[2], q, inside);
        if (l < best) { best = l; bq[0] = q[0]; bq[1] = q[1]; bq[2] = q[2]; bt = k; binside = inside; }
    }
    if (bt < 0 || !(best < 0.5f * R.thickness + R.margin)) return 0;
    if (binside) {
        const unsigned char* tv = R.shape.tris + 3 * bt;
        const float* a = R.shape.pts + 3 * tv[0];
        const float* b = R.shape.pts + 3 * tv[1];
        const float* c = R.shape.pts + 3 * tv[2];
        const float e0[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const float e1[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const float m0 = e0[1] * e1[2] - e0[2] * e1[1], m1 = e0[2] * e1[0] - e0[0] * e1[2],
                    m2 = e0[0] * e1[1] - e0[1] * e1[0];
        const float ln = sqrtf(m0 * m0 + m1 * m1 + m2 * m2);
        const float sg = ((p0 - bq[0]) * m0 + (p1 - bq[1]) * m1 + (p2 - bq[2]) * m2) >= 0.f ? 1.f : -1.f;
        nl[0] = sg * m0 / ln; nl[1] = sg * m1 / ln; nl[2] = sg * m2 / ln;
    } else if (best > 0.f) {
        nl[0] = (p0 - bq[0]) / best; nl[1] = (p1 - bq[1]) / best; nl[2] = (p2 - bq[2]) / best;
    }
    return 1;
}

// Region test of one rigid at world point x (Sec. IV).  Returns 0 none,
// 1 regular, 2 one-dimensional (segments), 3 sticky (slicer spine); n is the
// contact normal (zero when undefined) and t the 1D tangent.
// EXT: the launch has arcs or mesh slicers (a separate instance of the grid
// kernel, so that the common shapes keep their registers).
template <bool EXT>
__device__ int rigid_region(const RigidCur& R, float3 x, float3& n, float3& t)
{
    const float dx0 = x.x - R.c[0], dx1 = x.y - R.c[1], dx2 = x.z - R.c[2];
    // body coordinates p = R^T (x - c)
    const float p0 = R.R[0] * dx0 + R.R[3] * dx1 + R.R[6] * dx2;
    const float p1 = R.R[1] * dx0 + R.R[4] * dx1 + R.R[7] * dx2;
    const float p2 = R.R[2] * dx0 + R.R[5] * dx1 + R.R[8] * dx2;
    float nl0 = 0.f, nl1 = 0.f, nl2 = 0.f, tl0 = 0.f, tl1 = 0.f, tl2 = 0.f;
    int code = 0;
    if (R.type == MPM_SPHERE) {
        const float l = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
        if (l - R.radius < R.margin) {
            code = 1;
            if (l > 0.f) { nl0 = p0 / l; nl1 = p1 / l; nl2 = p2 / l; }
            else nl1 = 1.f;
        }
    } else if (R.type == MPM_BOX) {
        const float q0 = fabsf(p0) - R.half[0], q1 = fabsf(p1) - R.half[1], q2 = fabsf(p2) - R.half[2];
        const float o0 = fmaxf(q0, 0.f), o1 = fmaxf(q1, 0.f), o2 = fmaxf(q2, 0.f);
        const float out = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
        const float mx = fmaxf(q0, fmaxf(q1, q2));
        const float sdf = out + fminf(mx, 0.f);
        if (sdf < R.margin) {
            code = 1;
            if (out > 0.f) {
                nl0 = copysignf(o0 / out, p0);
                nl1 = copysignf(o1 / out, p1);
                nl2 = copysignf(o2 / out, p2);
                // copysignf(0, negative) gives -0: harmless
            } else if (q0 >= q1 && q0 >= q2) nl0 = p0 >= 0.f ? 1.f : -1.f;
            else if (q1 >= q2) nl1 = p1 >= 0.f ? 1.f : -1.f;
            else nl2 = p2 >= 0.f ? 1.f : -1.f;
        }
    } else if (R.type == MPM_QUAD_SLICER &&
               fabsf(p2) < (fmaxf(0.5f * R.thickness, R.spine_radius) + R.margin) * 1.000001f + 1e-30f) {
        // (beyond that distance from the blade plane neither the spine nor the faces
        // can hold the node: both distances are at least |p2|)
        const float A = R.half[0], Bh = R.half[1];
        const float es = fmaxf(fabsf(p0) - A, 0.f), et = p1 + Bh;
        const float dsp = sqrtf(es * es + et * et + p2 * p2);
        if (dsp < R.spine_radius + R.margin) {
            code = 3;
        } else {
            const float qs = fminf(fmaxf(p0, -A), A), qt = fminf(fmaxf(p1, -Bh), Bh);
            const float d0 = p0 - qs, d1 = p1 - qt, d2 = p2;
            const float l = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            if (l < 0.5f * R.thickness + R.margin) {
                code = 1;
                if (fabsf(p0) <= A && fabsf(p1) <= Bh) nl2 = p2 >= 0.f ? 1.f : -1.f;
                else { nl0 = d0 / l; nl1 = d1 / l; nl2 = d2 / l; }
            }
        }
    } else if (EXT && R.type == MPM_ARC) {
        // nearest point of the arc (radius half[0], angles half[1] .. half[1] + half[2])
        const float Ra = R.half[0], th0 = R.half[1], sw = R.half[2];
        const float kTwoPi = 6.28318530717958647f;
        float th = th0;
        if (p0 != 0.f || p1 != 0.f) {
            float rel = fmodf(atan2f(p1, p0) - th0, kTwoPi);
            if (rel < 0.f) rel += kTwoPi;
            if (rel <= sw) {
                th = th0 + rel;
            } else {
                float s0, c0, s1, c1;
                sincosf(th0, &s0, &c0);
                sincosf(th0 + sw, &s1, &c1);
                const float a0 = p0 - Ra * c0, a1 = p1 - Ra * s0, b0 = p0 - Ra * c1, b1 = p1 - Ra * s1;
                th = (b0 * b0 + b1 * b1 < a0 * a0 + a1 * a1) ? th0 + sw : th0;
            }
        }
        float sn, cs;
        sincosf(th, &sn, &cs);
        const float d0 = p0 - Ra * cs, d1 = p1 - Ra * sn, d2 = p2;
        const float l = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        if (l < R.radius + R.margin) {
            code = 2;
            if (l > 0.f) { nl0 = d0 / l; nl1 = d1 / l; nl2 = d2 / l; }
            tl0 = -sn;
            tl1 = cs;
        }
    } else if (EXT && R.type == MPM_MESH_SLICER) {
        float nl[3] = {0.f, 0.f, 0.f};
        code = mesh_slicer_region(R, p0, p1, p2, nl);
        nl0 = nl[0]; nl1 = nl[1]; nl2 = nl[2];
    } else if (R.type == MPM_SEGMENTS) {
        float best = 3.4e38f, bq0 = 0.f, bq1 = 0.f, bq2 = 0.f;
        int bs = -1;
        for (int s = 0; s + 1 < R.n_pts; ++s) {
            const float a0 = R.shape.pts[3 * s], a1 = R.shape.pts[3 * s + 1], a2 = R.shape.pts[3 * s + 2];
            const float e0 = R.shape.pts[3 * s + 3] - a0, e1 = R.shape.pts[3 * s + 4] - a1, e2 = R.shape.pts[3 * s + 5] - a2;
            const float L2 = e0 * e0 + e1 * e1 + e2 * e2;
            float u = L2 > 0.f ? ((p0 - a0) * e0 + (p1 - a1) * e1 + (p2 - a2) * e2) / L2 : 0.f;
            u = fminf(fmaxf(u, 0.f), 1.f);
            const float c0 = a0 + u * e0, c1 = a1 + u * e1, c2 = a2 + u * e2;
            const float d0 = p0 - c0, d1 = p1 - c1, d2 = p2 - c2;
            const float l = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            if (l < best) { best = l; bq0 = c0; bq1 = c1; bq2 = c2; bs = s; }
        }
        if (bs >= 0 && best < R.radius + R.margin) {
            code = 2;
            if (best > 0.f) { nl0 = (p0 - bq0) / best; nl1 = (p1 - bq1) / best; nl2 = (p2 - bq2) / best; }
            const float e0 = R.shape.pts[3 * bs + 3] - R.shape.pts[3 * bs], e1 = R.shape.pts[3 * bs + 4] - R.shape.pts[3 * bs + 1],
                        e2 = R.shape.pts[3 * bs + 5] - R.shape.pts[3 * bs + 2];
            const float L = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            if (L > 0.f) { tl0 = e0 / L; tl1 = e1 / L; tl2 = e2 / L; }
        }
    }
    n = f3(R.R[0] * nl0 + R.R[1] * nl1 + R.R[2] * nl2, R.R[3] * nl0 + R.R[4] * nl1 + R.R[5] * nl2,
           R.R[6] * nl0 + R.R[7] * nl1 + R.R[8] * nl2);
    t = f3(R.R[0] * tl0 + R.R[1] * tl1 + R.R[2] * tl2, R.R[3] * tl0 + R.R[4] * tl1 + R.R[5] * tl2,
           R.R[6] * tl0 + R.R[7] * tl1 + R.R[8] * tl2);
    return code;
}

// Contact correction (Sec. IV-A..C): sticky -> v_rel' = 0; otherwise keep a
// separating node (v_n >= 0), else v_rel' = c_d max(1 - mu_k |v_n| / |v_t|, 0) v_t
// with v_t the tangential part (regular) or the part along the 1D tangent.
// Returns whether the node was changed; dp = node momentum change.
template <bool EXT>
__device__ bool rigid_contact(const RigidCur& R, float3 x, float m, float3& v, float3& dp)
{
    float3 n, t;
    const int code = rigid_region<EXT>(R, x, n, t);
    if (code == 0) return false;
    const float r0 = x.x - R.c[0], r1 = x.y - R.c[1], r2 = x.z - R.c[2];
    const float vr0 = R.vel[0] + R.omega[1] * r2 - R.omega[2] * r1;
    const float vr1 = R.vel[1] + R.omega[2] * r0 - R.omega[0] * r2;
    const float vr2 = R.vel[2] + R.omega[0] * r1 - R.omega[1] * r0;
    const float e0 = v.x - vr0, e1 = v.y - vr1, e2 = v.z - vr2;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
    if (code != 3) {
        const bool has_n = (n.x * n.x + n.y * n.y + n.z * n.z) > 0.f;
        float vn = e0 * n.x + e1 * n.y + e2 * n.z;
        if (has_n && vn >= 0.f) return false;
        if (!has_n) vn = 0.f;
        float t0, t1, t2;
        if (code == 1) {
            t0 = e0 - vn * n.x; t1 = e1 - vn * n.y; t2 = e2 - vn * n.z;
        } else {
            const float a = e0 * t.x + e1 * t.y + e2 * t.z;
            t0 = a * t.x; t1 = a * t.y; t2 = a * t.z;
        }
        const float lt = sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
        float scale = 0.f;
        if (lt > 0.f) scale = R.c_d * fmaxf(1.f - R.mu_k * fabsf(vn) / lt, 0.f);
        n0 = scale * t0; n1 = scale * t1; n2 = scale * t2;
    }
    dp = f3(m * (n0 - e0), m * (n1 - e1), m * (n2 - e2));
    v = f3(vr0 + n0, vr1 + n1, vr2 + n2);
    return true;
}

__device__ void stage_rigid(const RigidDev& src, double t_now, RigidCur& dst)
{
    dst.type = src.type;
    dst.n_pts = src.n_pts;
    dst.n_tris = src.n_tris;
    dst.n_spine = src.n_spine;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dst.vel[i] = src.vel[i];
        dst.omega[i] = src.omega[i];
        dst.half[i] = src.half[i];
    }
    rigid_pose_at(src, t_now, dst.c, dst.R);
    dst.mu_k = src.mu_k;
    dst.c_d = src.c_d;
    dst.margin = src.margin;
    dst.radius = src.radius;
    dst.thickness = src.thickness;
    dst.spine_radius = src.spine_radius;
}

constexpr int kGridThreads = 256;  // 4 node bricks per iteration

__device__ void flush_impulse(const StepArgs& a, const float* simp, int scene, int nr, int tid)
{
    for (int t = tid; t < nr * 6; t += kGridThreads)
        if (simp[t] != 0.f) atomicAdd(&a.impulse[scene * kMaxRigids * 6 + t], (double)simp[t]);
}

// Grid update of the active node bricks: 64 threads per brick, one node each.
// Rigids of a scene are staged in shared memory (posed at the scene's clock).
// Grid update of node nid of node brick B (Eq. 3, contact, walls), clearing
// the P2G accumulator; rigid impulses are summed into simp (shared).
// The node's P2G accumulator is reset afterwards by k_grid_clear: loading and
// clearing the freshly reduced lines in one kernel measured far slower.
template <bool EXT>
__device__ __forceinline__ void grid_node(const StepArgs& a, int B, int scene, int nid, int lane, const RigidCur* rig,
                                          int nr, float* simp)
{
    const SceneDev sc = a.scenes[scene];
    const int n = sc.n, lb = B - sc.brick_base;
    int bx, by, bz;
    brick_coords(sc.nb, sc.nb_log2, lb, bx, by, bz);
    const int gi = bx * 4 + (nid >> 4);
    const int gj = by * 4 + ((nid >> 2) & 3);
    const int gk = bz * 4 + (nid & 3);
    const int node = B * 64 + nid;
    const float4 g = a.G[node];
    float3 v = f3(0.f, 0.f, 0.f);
    const float dxs = 1.0f / (float)n;
    float dpr[kMaxRigids][3];
    unsigned touched = 0;
    if (g.x > 0.f) {
        v = f3(g.y / g.x + a.dt * a.gravity[0], g.z / g.x + a.dt * a.gravity[1], g.w / g.x + a.dt * a.gravity[2]);
        const float3 xI = f3(gi * dxs, gj * dxs, gk * dxs);
        for (int r = 0; r < nr; ++r) {
            float3 dp;
            if (rigid_contact<EXT>(rig[r], xI, g.x, v, dp)) {
                touched |= 1u << r;
                dpr[r][0] = dp.x; dpr[r][1] = dp.y; dpr[r][2] = dp.z;
            }
        }
        const int lo = a.bound, hi = n - 1 - a.bound;
        if (gi < lo) v.x = fmaxf(v.x, 0.f);
        if (gi > hi) v.x = fminf(v.x, 0.f);
        if (gj < lo) {
            if (a.floor_sticky) v = f3(0.f, 0.f, 0.f);
            else v.y = fmaxf(v.y, 0.f);
        }
        if (gj > hi) v.y = fminf(v.y, 0.f);
        if (gk < lo) v.z = fmaxf(v.z, 0.f);
        if (gk > hi) v.z = fminf(v.z, 0.f);
    }
    a.V[node] = make_float4(v.x, v.y, v.z, g.x);
    if (nid == 0) {
        a.brick_epoch[B] = a.epoch[scene];
        // the histogram of the next substep starts from zero (the scan has
        // read it; every non-empty brick is an active node brick)
        a.sb.cnt[B] = 0;
    }
    // impulse on each rigid: -(node momentum change), linear and angular
    for (int r = 0; r < nr; ++r) {
        const bool on = (touched >> r) & 1u;
        if (!__any_sync(kFull, on)) continue;
        float val[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (on) {
            const float d0 = -dpr[r][0], d1 = -dpr[r][1], d2 = -dpr[r][2];
            const float r0 = gi * dxs - rig[r].c[0], r1 = gj * dxs - rig[r].c[1], r2 = gk * dxs - rig[r].c[2];
            val[0] = d0; val[1] = d1; val[2] = d2;
            val[3] = r1 * d2 - r2 * d1;
            val[4] = r2 * d0 - r0 * d2;
            val[5] = r0 * d1 - r1 * d0;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float x = val[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            if (lane == 0) atomicAdd(&simp[r * 6 + c], x);
        }
    }
}

// Grid update of a launch whose scenes have no rigid: no staging and no impulse
// sums, so a budget of 32 registers holds twice the resident CTAs of k_grid and
// the node bricks of a 1M-particle block are taken in one round.
__global__ void __launch_bounds__(kGridThreads, 8) k_grid_plain(StepArgs a)
{
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 6, nid = tid & 63;
    const int n_nact = a.sb.counters[CTR_N_NACT];
    for (int base = blockIdx.x * 4; base < n_nact; base += gridDim.x * 4) {
        const int item = base + grp;
        if (item < n_nact)
            grid_node<false>(a, a.sb.nact_brick[item], a.sb.nact_scene[item], nid, lane, nullptr, 0, nullptr);
    }
}

// Reset of the P2G accumulator and of the node-brick flags of the active node
// bricks once the grid update and the scan have read them.  Loading and clearing the lines that P2G's reductions just wrote
// in one kernel measured far slower than two kernels: 13.4 against 11.5 us per
// substep for the 1M block without rigids, 0.138 against 0.047 ms for the 256
// batched scenes with their blades.
__global__ void __launch_bounds__(kGridThreads, 8) k_grid_clear(StepArgs a)
{
    const int grp = threadIdx.x >> 6, nid = threadIdx.x & 63;
    const int n_nact = a.sb.counters[CTR_N_NACT];
    for (int base = blockIdx.x * 4; base < n_nact; base += gridDim.x * 4) {
        const int item = base + grp;
        if (item < n_nact) {
            const int B = a.sb.nact_brick[item];
            a.G[B * 64 + nid] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nid == 0) a.sb.nflag[B] = 0;  // the scan has read it (resetting it there was slower)
        }
    }
}

template <bool EXT>
__global__ void __launch_bounds__(kGridThreads, 4) k_grid(StepArgs a)
{
    __shared__ RigidCur rig[kMaxRigids];
    __shared__ float simp[kMaxRigids * 6];
    // per brick of a chunk of the list: node brick, scene, the scene's rigid count
    __shared__ int s_brk[kGridThreads], s_scn[kGridThreads], s_nr[kGridThreads];
    __shared__ int s_scene[4];
    __shared__ int s_staged, s_nrig, s_target;
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 6, nid = tid & 63;
    const int n_nact = a.sb.counters[CTR_N_NACT];
    if (!a.any_rigid) {
        // no scene has a rigid: 4 node bricks per step, no staging, no barriers
        for (int base = blockIdx.x * 4; base < n_nact; base += gridDim.x * 4) {
            const int item = base + grp;
            if (item < n_nact) grid_node<EXT>(a, a.sb.nact_brick[item], a.sb.nact_scene[item], nid, lane, nullptr, 0, nullptr);
        }
        return;
    }
    if (tid == 0) { s_staged = -1; s_nrig = 0; }
    // each CTA takes a contiguous run of the node-brick list (scenes are contiguous
    // in it), so that it stages a scene's rigids and flushes their impulses about
    // once; groups of 4 bricks of the staged scene (or of scenes without rigids)
    // then run without barriers
    const int per = ((n_nact + gridDim.x - 1) / gridDim.x + 3) & ~3;
    const int first = blockIdx.x * per, last = min(first + per, n_nact);
    for (int c0 = first; c0 < last; c0 += kGridThreads) {
        const int c1 = min(c0 + kGridThreads, last);
        __syncthreads();  // the previous chunk's table is no longer read
        if (c0 + tid < c1) {
            const int sc = a.sb.nact_scene[c0 + tid];
            s_brk[tid] = a.sb.nact_brick[c0 + tid];
            s_scn[tid] = sc;
            s_nr[tid] = a.scenes[sc].n_rigid;
        }
        __syncthreads();
        for (int base = c0; base < c1; base += 4) {
            const int item = base + grp;
            const int my_scene = item < c1 ? s_scn[item - c0] : -1;
            const int gl = min(base + 3, c1 - 1) - c0;
            bool no_rigid = true, staged = true;
            for (int g = base - c0; g <= gl; ++g) {
                no_rigid = no_rigid && s_nr[g] == 0;
                staged = staged && s_scn[g] == s_staged;
            }
            const int my_brick = my_scene >= 0 ? s_brk[item - c0] : 0;
            if (no_rigid) {
                if (my_scene >= 0) grid_node<EXT>(a, my_brick, my_scene, nid, lane, nullptr, 0, nullptr);
                continue;
            }
            if (staged) {
                if (my_scene >= 0) grid_node<EXT>(a, my_brick, my_scene, nid, lane, rig, s_nrig, simp);
                continue;
            }
            if (nid == 0) s_scene[grp] = my_scene;
            bool done = my_scene < 0;
            __syncthreads();
            for (;;) {
                // next scene to process among the 4 bricks (usually all the same)
                if (tid == 0) {
                    int t = -1;
                    for (int g = 0; g < 4; ++g)
                        if (s_scene[g] >= 0 && (t < 0 || s_scene[g] < t)) t = s_scene[g];
                    s_target = t;
                }
                __syncthreads();
                const int target = s_target;
                if (target < 0) break;
                if (target != s_staged) {
                    if (s_staged >= 0) flush_impulse(a, simp, s_staged, s_nrig, tid);
                    __syncthreads();
                    const int nr = a.scenes[target].n_rigid;
                    const double t_now = a.t_scene[target];
                    if (tid < nr) stage_rigid(a.rigids[target * kMaxRigids + tid], t_now, rig[tid]);
                    constexpr int kShapeWords = (int)(sizeof(RigidShape) / sizeof(int));
                    static_assert(sizeof(RigidShape) % sizeof(int) == 0, "shape copied in words");
                    for (int t = tid; t < nr * kShapeWords; t += kGridThreads) {
                        const int r = t / kShapeWords, k = t % kShapeWords;
                        reinterpret_cast<int*>(&rig[r].shape)[k] =
                            reinterpret_cast<const int*>(&a.rigids[target * kMaxRigids + r].shape)[k];
                    }
                    for (int t = tid; t < kMaxRigids * 6; t += kGridThreads) simp[t] = 0.f;
                    if (tid == 0) { s_staged = target; s_nrig = nr; }
                    __syncthreads();
                }
                if (!done && my_scene == target) {
                    done = true;
                    grid_node<EXT>(a, my_brick, target, nid, lane, rig, s_nrig, simp);
                }
                __syncthreads();
                if (nid == 0 && my_scene == target) s_scene[grp] = -1;
                __syncthreads();
            }
        }
    }
    __syncthreads();
    if (s_staged >= 0) flush_impulse(a, simp, s_staged, s_nrig, tid);
}

// ------------------------------------------------------------------ G2P
//
// One CTA per active particle brick.  The 2x2x2 node bricks holding the 6^3
// velocity window are staged in shared memory by bulk-copy TMA, double
// buffered: the next brick's window is in flight while this brick computes.

// G2P of one particle from the staged window (Eq. 4, Eq. 9, Eq. 10) followed by
// the constitutive update (the last step of the G2P loop in Algorithm 1).
// Writes x, v, C, F (and id, mu, lam) to slot s of the output state; returns
// the new position, velocity, C and the Kirchhoff stress of the new F.
struct G2POut {
    float x[3], v[3], C[9], t6[6];
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Staged mode (sX != nullptr): x and F of particle p were copied into
// sX[d * stride] and sF[q * stride] by cp.async one particle ahead; this call
// starts the copies of particle pnext (when >= 0) as soon as its own values
// are out of the buffers: x after the gather, F after the F update.
// Variants of the forward G2P (template flags).
enum {
    kG2PSolids = 1,    // push particles out of solid rigids (some scene has a rigid)
    kG2PStdGrad = 2,   // standard MPM: L = sum v_I grad phi^T instead of the APIC C (Eq. 5)
    kG2PNoStress = 4   // PB-MPM: no constitutive update (no stress is stored)
};

// The new position is returned in o.x and stored by the caller, after the
// particle push-out (finish_position).
template <int FLAGS>
__device__ __forceinline__ unsigned g2p_particle(const StepArgs& a, const SceneDev& sc, const float4* lin, int p, int s,
                                                 int ox, int oy, int oz, G2POut& o, float* sX = nullptr,
                                                 float* sF = nullptr, int stride = 0, int pnext = -1,
                                                 int* sI = nullptr)
{
    const int cap = a.cap, n = sc.n;
    const float fn = (float)n, dt = a.dt;
    unsigned ebits = 0;
    if (sX) cp_async_wait_all();
    const float x0 = sX ? sX[0] : a.in.x[p], x1 = sX ? sX[stride] : a.in.x[cap + p],
                x2 = sX ? sX[2 * stride] : a.in.x[2 * cap + p];
    const int id_staged = sI ? sI[0] : 0;  // read before the next particle's copy lands
    int bc[3];
    float f[3], w[9];
    particle_weights(x0, x1, x2, n, bc, f, w);
    const int l0 = min(max(bc[0] - ox, 0), 3), l1 = min(max(bc[1] - oy, 0), 3), l2 = min(max(bc[2] - oz, 0), 3);
    // separable contraction over k, then j, then i of
    //   v = sum W v_I,  B_rc = sum W v_I,r (o_c - f_c),  W = wx_i wy_j wz_k
    const float* wx = w;
    const float* wy = w + 3;
    const float* wz = w + 6;
    float wxd[3], wyd[3], wzd[3];
    if (FLAGS & kG2PStdGrad) {
        // the basis gradient in cell units (times n below): L_rc = n sum v_r dW/df_c
        bspline_d(f[0], wxd);
        bspline_d(f[1], wyd);
        bspline_d(f[2], wzd);
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            wxd[q] = wx[q] * ((float)q - f[0]);
            wyd[q] = wy[q] * ((float)q - f[1]);
            wzd[q] = wz[q] * ((float)q - f[2]);
        }
    }
    const float4* base = lin + (l0 * 36 + l1 * 6 + l2);
    float A[3][3], Ay[3][3], Bz[3][3];  // [i][component]
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int c = 0; c < 3; ++c) A[i][c] = Ay[i][c] = Bz[i][c] = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float4 g0 = base[i * 36 + j * 6], g1 = base[i * 36 + j * 6 + 1], g2 = base[i * 36 + j * 6 + 2];
            const float ax = wz[0] * g0.x + wz[1] * g1.x + wz[2] * g2.x;
            const float ay = wz[0] * g0.y + wz[1] * g1.y + wz[2] * g2.y;
            const float az = wz[0] * g0.z + wz[1] * g1.z + wz[2] * g2.z;
            const float bx = wzd[0] * g0.x + wzd[1] * g1.x + wzd[2] * g2.x;
            const float by = wzd[0] * g0.y + wzd[1] * g1.y + wzd[2] * g2.y;
            const float bz = wzd[0] * g0.z + wzd[1] * g1.z + wzd[2] * g2.z;
            A[i][0] += wy[j] * ax; A[i][1] += wy[j] * ay; A[i][2] += wy[j] * az;
            Ay[i][0] += wyd[j] * ax; Ay[i][1] += wyd[j] * ay; Ay[i][2] += wyd[j] * az;
            Bz[i][0] += wy[j] * bx; Bz[i][1] += wy[j] * by; Bz[i][2] += wy[j] * bz;
        }
    }
    float vv[3], B[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        vv[r] = wx[0] * A[0][r] + wx[1] * A[1][r] + wx[2] * A[2][r];
        B[3 * r] = wxd[0] * A[0][r] + wxd[1] * A[1][r] + wxd[2] * A[2][r];
        B[3 * r + 1] = wx[0] * Ay[0][r] + wx[1] * Ay[1][r] + wx[2] * Ay[2][r];
        B[3 * r + 2] = wx[0] * Bz[0][r] + wx[1] * Bz[1][r] + wx[2] * Bz[2][r];
    }
    const float v0 = vv[0], v1 = vv[1], v2 = vv[2];
    if (sX && pnext >= 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) cp_async4(sX + d * stride, a.in.x + (size_t)d * cap + pnext);
        if (sI) cp_async4(reinterpret_cast<float*>(sI), reinterpret_cast<const float*>(a.in.id + pnext));
    }
    // C = D^-1 sum N v (x_I - x_p)^T = 4/dx^2 * dx * B  (Eq. 9), or for the
    // standard MPM L = n B with the derivative weights (Eq. 5); x += dt v (Eq. 4)
    const float c4 = (FLAGS & kG2PStdGrad) ? fn : 4.0f * fn;
#pragma unroll
    for (int i = 0; i < 9; ++i) o.C[i] = B[i] * c4;
    o.v[0] = v0; o.v[1] = v1; o.v[2] = v2;
    o.x[0] = x0 + dt * v0;
    o.x[1] = x1 + dt * v1;
    o.x[2] = x2 + dt * v2;
#pragma unroll
    for (int d = 0; d < 3; ++d) a.out.v[(size_t)d * cap + s] = o.v[d];
#pragma unroll
    for (int i = 0; i < 9; ++i) a.out.C[(size_t)i * cap + s] = o.C[i];
    a.out.id[s] = sI ? id_staged : a.in.id[p];
    float mu, lam;
    if (sc.pp_mat) {
        mu = a.in.mu[p];
        lam = a.in.lam[p];
        a.out.mu[s] = mu;
        a.out.lam[s] = lam;
    } else {
        mu = sc.mu;
        lam = sc.lam;
    }
    // F <- (I + dt C) F  (Eq. 10)
    float Fn[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float F0 = sF ? sF[c * stride] : a.in.F[(size_t)c * cap + p];
        const float F1 = sF ? sF[(3 + c) * stride] : a.in.F[(size_t)(3 + c) * cap + p];
        const float F2 = sF ? sF[(6 + c) * stride] : a.in.F[(size_t)(6 + c) * cap + p];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float Fr = r == 0 ? F0 : (r == 1 ? F1 : F2);
            Fn[3 * r + c] = Fr + dt * (o.C[3 * r] * F0 + o.C[3 * r + 1] * F1 + o.C[3 * r + 2] * F2);
        }
    }
    if (sF && pnext >= 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) cp_async4(sF + q * stride, a.in.F + (size_t)q * cap + pnext);
    }
    if (!(FLAGS & kG2PNoStress)) ebits |= constitutive(a.model, a.plasticity, a.yield_stress, mu, lam, Fn, o.t6);
#pragma unroll
    for (int i = 0; i < 9; ++i) a.out.F[(size_t)i * cap + s] = Fn[i];
    float chk = x0 + x1 + x2 + v0 + v1 + v2;
#pragma unroll
    for (int i = 0; i < 9; ++i) chk += Fn[i];
    if (!isfinite(chk)) ebits |= MPM_EBIT_NONFINITE;
    return ebits;
}

// Push-out against the scene's solid rigids at the end of the substep
// (n_solid = 0: none), then the position store at slot s.
__device__ __forceinline__ void finish_position(const StepArgs& a, const SolidPose* poses, int n_solid, int s,
                                                float x[3])
{
    if (n_solid) push_out(poses, n_solid, x);
#pragma unroll
    for (int d = 0; d < 3; ++d) a.out.x[(size_t)d * a.cap + s] = x[d];
}

// Copy the 6^3 window out of the 2x2x2 staged bricks into a linear array, so
// that the 27 nodes of a particle sit at constant offsets.
template <int BLOCK>
__device__ __forceinline__ void linearize_window(const float4* vw, float4* lin)
{
    for (int t = threadIdx.x; t < kWinNodes; t += BLOCK) {
        const int wi = t / 36, wj = (t / 6) % 6, wk = t % 6;
        lin[t] = vw[(((wi >> 2) << 2) | ((wj >> 2) << 1) | (wk >> 2)) * 64 + (wi & 3) * 16 + (wj & 3) * 4 + (wk & 3)];
    }
}

// MINB = CTAs per SM the registers must allow: the larger budget (7 at 128
// threads, 72 registers; 3 at 256, 80; 1 at 512) or 1024/BLOCK (64 registers,
// more warps in flight).  SOLIDS: some scene of the launch has a sphere or a
// box, so particles may need the push-out (a separate variant: its extra live
// registers would make the plain build spill).
template <int BLOCK, int MINB, int FLAGS>
__global__ void __launch_bounds__(BLOCK, MINB) k_g2p(StepArgs a)
{
    constexpr bool SOLIDS = (FLAGS & kG2PSolids) != 0;
    // x, F and (with 72 or more registers; the 64-register builds would spill) the
    // id of each thread's next particle, copied by cp.async one particle ahead
    constexpr bool STAGE_ID = 65536 / (BLOCK * MINB) >= 72;
    __shared__ float sX[3 * BLOCK], sF[9 * BLOCK];
    __shared__ int sI[STAGE_ID ? BLOCK : 1];
    __shared__ __align__(128) float4 vw[2][8 * 64];
    __shared__ __align__(16) float4 lin[kWinNodes];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_item[2];
    __shared__ SolidPose s_pose[kMaxRigids];  // the scene's rigids at the end of the substep
    __shared__ int s_pose_scene;
    const int tid = threadIdx.x;
    const int n_act = a.sb.counters[CTR_N_ACT];
    int* work = &a.sb.counters[CTR_WORK_G2P];
    if (tid == 0) s_pose_scene = -1;
    walker_init<BLOCK>(a, n_act, vw, bar, s_item, work);
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    for (;;) {
        const int item = s_item[buf];
        if (item >= n_act) break;
        if (!walker_next(a, n_act, vw, bar, s_item, work, buf, phase, item)) break;
        const int start = a.sb.act_start[item], count = a.sb.act_count[item], scene = a.sb.act_scene[item];
        const SceneDev sc = a.scenes[scene];
        // s_pose_scene changes only after the barrier below, which every thread
        // passes after this test
        const int n_solid = SOLIDS ? sc.n_rigid : 0;
        if (n_solid && scene != s_pose_scene) stage_solids(a, scene, s_pose);
        const int nb = sc.nb, lb = a.sb.act_brick[item] - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        // the brick's first particle of each thread: its copies start here (the
        // thread's last call of the previous brick has read both buffers)
        int pcur = tid < count ? a.sb.perm[start + tid] : -1;
        if (pcur >= 0) {
#pragma unroll
            for (int d = 0; d < 3; ++d) cp_async4(&sX[d * BLOCK + tid], a.in.x + (size_t)d * a.cap + pcur);
#pragma unroll
            for (int q = 0; q < 9; ++q) cp_async4(&sF[q * BLOCK + tid], a.in.F + (size_t)q * a.cap + pcur);
            if (STAGE_ID) cp_async4(reinterpret_cast<float*>(&sI[tid]), reinterpret_cast<const float*>(a.in.id + pcur));
        }
        linearize_window<BLOCK>(vw[buf], lin);
        __syncthreads();
        if (tid == 0 && n_solid) s_pose_scene = scene;
        unsigned ebits = 0;
        for (int k0 = 0; k0 < count; k0 += BLOCK) {
            const int k = k0 + tid;
            const bool valid = k < count;
            int key = 0;
            if (valid) {
                G2POut o;
                const int pnext = k + BLOCK < count ? a.sb.perm[start + k + BLOCK] : -1;
                ebits |= g2p_particle<FLAGS>(a, sc, lin, pcur, start + k, ox, oy, oz, o, &sX[tid], &sF[tid], BLOCK,
                                             pnext, STAGE_ID ? &sI[tid] : nullptr);
                pcur = pnext;
                if (!(FLAGS & kG2PNoStress))
#pragma unroll
                    for (int q = 0; q < 6; ++q) a.out.tau[(size_t)q * a.cap + start + k] = o.t6[q];
                finish_position(a, SOLIDS ? s_pose : nullptr, n_solid, start + k, o.x);
                unsigned ood = 0;
                key = cell_key(sc, o.x[0], o.x[1], o.x[2], ood);
                if (ood && !(ebits & MPM_EBIT_NONFINITE)) ebits |= MPM_EBIT_OUT_OF_DOMAIN;
            }
            const int rank = aggregated_rank_mark(a.sb, sc, key >> 6, valid);
            if (valid) {
                a.sb.key[start + k] = key;
                a.sb.rank[start + k] = rank;
            }
        }
        if (ebits) atomicOr(&a.err[scene], ebits);
        __syncthreads();
        buf ^= 1;
    }
    walker_exit(a);
}

// ------------------------------------------------------- fused G2P + P2G
//
// G2P of substep k fused with P2G of substep k+1: each particle is read and
// written once per substep, and its new stress goes from registers straight
// into the next P2G.  The CTA of a brick scatters into an 8^3-node window
// around the brick (base cells may have moved by up to one cell): particles
// whose new base cell is still inside the brick use the per-cell register
// accumulation of k_p2g; the few that crossed a brick face use shared atomics
// into the window; any that moved farther use global atomics.

constexpr int kFusedThreads = 192;  // 64 cells x 3 slices
constexpr int kW8 = 8, kW8Nodes = kW8 * kW8 * kW8;

__global__ void __launch_bounds__(kFusedThreads, 4) k_g2p2g(StepArgs a)
{
    __shared__ __align__(128) float4 vw[2][8 * 64];
    __shared__ __align__(16) float4 lin[kWinNodes];
    __shared__ float rec[kRecFields][kFusedThreads];
    __shared__ float win[4][kW8Nodes];
    __shared__ short order[kFusedThreads];
    __shared__ int cell_cnt[64], cell_off[65];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_item[2];
    __shared__ SolidPose s_pose[kMaxRigids];  // the scene's rigids at the end of the substep
    __shared__ int s_pose_scene;
    const int tid = threadIdx.x;
    const int cell = tid & 63, slice = tid >> 6;
    const int cx = cell >> 4, cy = (cell >> 2) & 3, cz = cell & 3;
    const int n_act = a.sb.counters[CTR_N_ACT];
    int* work = &a.sb.counters[CTR_WORK_G2P];
    if (tid == 0) s_pose_scene = -1;
    walker_init<kFusedThreads>(a, n_act, vw, bar, s_item, work);
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    for (;;) {
        const int item = s_item[buf];
        if (item >= n_act) break;
        for (int t = tid; t < 4 * kW8Nodes; t += kFusedThreads) (&win[0][0])[t] = 0.0f;
        if (tid < 64) cell_cnt[tid] = 0;
        if (!walker_next(a, n_act, vw, bar, s_item, work, buf, phase, item)) break;
        const int start = a.sb.act_start[item], count = a.sb.act_count[item], scene = a.sb.act_scene[item];
        const SceneDev sc = a.scenes[scene];
        const int n_solid = a.any_solid ? sc.n_rigid : 0;
        if (n_solid && scene != s_pose_scene) stage_solids(a, scene, s_pose);
        const int n = sc.n, nb = sc.nb, lb = a.sb.act_brick[item] - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float fn = (float)n, dxs = 1.0f / fn;
        const float m = sc.m_p;
        const float kA = a.dt * sc.V0 * 4.0f * fn * fn;
        linearize_window<kFusedThreads>(vw[buf], lin);
        __syncthreads();
        if (tid == 0 && n_solid) s_pose_scene = scene;
        unsigned ebits = 0;
        for (int k0 = 0; k0 < count; k0 += kFusedThreads) {
            const int k = k0 + tid;
            const bool valid = k < count;
            int key = 0, my_cell = -1, my_rank = 0;
            if (valid) {
                G2POut o;
                ebits |= g2p_particle<0>(a, sc, lin, a.sb.perm[start + k], start + k, ox, oy, oz, o);
                finish_position(a, s_pose, n_solid, start + k, o.x);
                // P2G of the next substep at the new position
                int bc[3];
                float f[3], w[9];
                const unsigned ood = particle_weights(o.x[0], o.x[1], o.x[2], n, bc, f, w);
                if (ood && !(ebits & MPM_EBIT_NONFINITE)) ebits |= ood;
                key = (sc.brick_base + ((bc[0] >> 2) * nb + (bc[1] >> 2)) * nb + (bc[2] >> 2)) * 64 +
                      ((bc[0] & 3) * 16 + (bc[1] & 3) * 4 + (bc[2] & 3));
                float q3[3], Ad[9];
                p2g_coeffs(m, kA, dxs, o.v, o.C, o.t6, f, q3, Ad);
                const int l0 = bc[0] - ox, l1 = bc[1] - oy, l2 = bc[2] - oz;
                if ((unsigned)l0 < 4u && (unsigned)l1 < 4u && (unsigned)l2 < 4u) {
                    put_record<kFusedThreads>(rec, tid, w, q3, Ad);
                    my_cell = (l0 * 4 + l1) * 4 + l2;
                    my_rank = atomicAdd(&cell_cnt[my_cell], 1);
                } else if (l0 >= -1 && l0 <= 4 && l1 >= -1 && l1 <= 4 && l2 >= -1 && l2 <= 4) {
                    // crossed a brick face: scatter into the window with shared atomics
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2) {
                                const float W = w[i] * w[3 + j] * w[6 + k2];
                                const int node = ((l0 + 1 + i) * kW8 + (l1 + 1 + j)) * kW8 + (l2 + 1 + k2);
                                atomicAdd(&win[0][node], W * m);
                                atomicAdd(&win[1][node], W * (q3[0] + Ad[0] * i + Ad[1] * j + Ad[2] * k2));
                                atomicAdd(&win[2][node], W * (q3[1] + Ad[3] * i + Ad[4] * j + Ad[5] * k2));
                                atomicAdd(&win[3][node], W * (q3[2] + Ad[6] * i + Ad[7] * j + Ad[8] * k2));
                            }
                } else {
                    // moved more than a cell: straight to HBM
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2) {
                                const float W = w[i] * w[3 + j] * w[6 + k2];
                                red_add_v4(&a.G[node_index(sc, bc[0] + i, bc[1] + j, bc[2] + k2)], W * m,
                                           W * (q3[0] + Ad[0] * i + Ad[1] * j + Ad[2] * k2),
                                           W * (q3[1] + Ad[3] * i + Ad[4] * j + Ad[5] * k2),
                                           W * (q3[2] + Ad[6] * i + Ad[7] * j + Ad[8] * k2));
                            }
                }
            }
            const int rank = aggregated_rank_mark(a.sb, sc, key >> 6, valid);
            if (valid) {
                a.sb.key[start + k] = key;
                a.sb.rank[start + k] = rank;
            }
            __syncthreads();
            scan_cells(cell_cnt, cell_off, tid);
            __syncthreads();
            if (my_cell >= 0) order[cell_off[my_cell] + my_rank] = (short)tid;
            __syncthreads();
            float acc_w[9], acc_p[9][3];
#pragma unroll
            for (int q = 0; q < 9; ++q) { acc_w[q] = 0.f; acc_p[q][0] = acc_p[q][1] = acc_p[q][2] = 0.f; }
            cell_accumulate<kFusedThreads>(rec, order, cell_off[cell], cell_off[cell + 1], slice, acc_w, acc_p);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (acc_w[q] != 0.f) {
                    const int node = ((cx + 1 + slice) * kW8 + (cy + 1 + q / 3)) * kW8 + (cz + 1 + q % 3);
                    atomicAdd(&win[0][node], acc_w[q] * m);
                    atomicAdd(&win[1][node], acc_p[q][0]);
                    atomicAdd(&win[2][node], acc_p[q][1]);
                    atomicAdd(&win[3][node], acc_p[q][2]);
                }
            }
            __syncthreads();
            if (tid < 64) cell_cnt[tid] = 0;
            __syncthreads();
        }
        // window -> HBM (node (ox-1, oy-1, oz-1) + (wi, wj, wk))
        for (int t = tid; t < kW8Nodes; t += kFusedThreads) {
            const float mm = win[0][t];
            if (mm == 0.0f) continue;
            const int gi = ox - 1 + t / (kW8 * kW8), gj = oy - 1 + (t / kW8) % kW8, gk = oz - 1 + t % kW8;
            if (gi < 0 || gj < 0 || gk < 0 || gi >= n || gj >= n || gk >= n) continue;
            red_add_v4(&a.G[node_index(sc, gi, gj, gk)], mm, win[1][t], win[2][t], win[3][t]);
        }
        if (ebits) atomicOr(&a.err[scene], ebits);
        __syncthreads();
        buf ^= 1;
    }
    walker_exit(a);
}

// ------------------------------------------------------- standard MPM P2G
//
// P2G of the standard MPM (Sec. III-A): m_I += W m (Eq. 1), and the momentum
// W m v plus the internal-force impulse -dt V0 tau grad W (Eq. 2, 3; V sigma =
// V0 tau).  One CTA per active particle brick accumulates its 6^3 window with
// shared-memory float atomics and adds it to HBM with one vector reduction per
// node.  The paper keeps this solver as a reference with fewer features; so
// does this kernel (no per-cell work items).

constexpr int kStdThreads = 256;

__global__ void __launch_bounds__(kStdThreads) k_p2g_std(StepArgs a)
{
    __shared__ float win[4][kWinNodes];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const int n_act = a.sb.counters[CTR_N_ACT];
    const int cap = a.cap;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.sb.counters[CTR_WORK_P2G], 1);
        for (int t = tid; t < 4 * kWinNodes; t += kStdThreads) (&win[0][0])[t] = 0.0f;
        __syncthreads();
        const int item = s_item;
        if (item >= n_act) break;
        const int b = a.sb.act_brick[item], start = a.sb.act_start[item], count = a.sb.act_count[item];
        const int scene = a.sb.act_scene[item];
        const SceneDev sc = a.scenes[scene];
        const int n = sc.n, nb = sc.nb, lb = b - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float fn = (float)n, m = sc.m_p;
        const float kap = a.dt * sc.V0 * fn;  // dt V0 times the n of grad W = n dW/df
        unsigned ebits = 0;
        for (int k = tid; k < count; k += kStdThreads) {
            const int p = a.sb.perm[start + k];
            int bc[3];
            float f[3], w[9], dw[9];
            ebits |= particle_weights(a.in.x[p], a.in.x[cap + p], a.in.x[2 * cap + p], n, bc, f, w);
            bspline_d(f[0], dw);
            bspline_d(f[1], dw + 3);
            bspline_d(f[2], dw + 6);
            float t6[6], v[3];
            if (a.tau_valid) {
#pragma unroll
                for (int q = 0; q < 6; ++q) t6[q] = a.in.tau[(size_t)q * cap + p];
            } else {
                float F[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) F[q] = a.in.F[(size_t)q * cap + p];
                const float mu = sc.pp_mat ? a.in.mu[p] : sc.mu, lam = sc.pp_mat ? a.in.lam[p] : sc.lam;
                ebits |= constitutive(a.model, 0, 0.f, mu, lam, F, t6);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] = m * a.in.v[(size_t)q * cap + p];
            const float tau[9] = {t6[0], t6[1], t6[2], t6[1], t6[3], t6[4], t6[2], t6[4], t6[5]};
            const int l0 = min(max(bc[0] - ox, 0), 3), l1 = min(max(bc[1] - oy, 0), 3), l2 = min(max(bc[2] - oz, 0), 3);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) {
                        const float W = w[i] * w[3 + j] * w[6 + kk];
                        const float g0 = dw[i] * w[3 + j] * w[6 + kk], g1 = w[i] * dw[3 + j] * w[6 + kk],
                                    g2 = w[i] * w[3 + j] * dw[6 + kk];
                        const int node = (l0 + i) * 36 + (l1 + j) * 6 + (l2 + kk);
                        atomicAdd(&win[0][node], W * m);
#pragma unroll
                        for (int r = 0; r < 3; ++r)
                            atomicAdd(&win[1 + r][node],
                                      W * v[r] - kap * (tau[3 * r] * g0 + tau[3 * r + 1] * g1 + tau[3 * r + 2] * g2));
                    }
        }
        __syncthreads();
        for (int q = tid; q < kWinNodes; q += kStdThreads) {
            const float mm = win[0][q];
            if (mm == 0.0f) continue;
            const int gi = ox + q / 36, gj = oy + (q / 6) % 6, gk = oz + q % 6;
            if (gi >= n || gj >= n || gk >= n) continue;
            red_add_v4(&a.G[node_index(sc, gi, gj, gk)], mm, win[1][q], win[2][q], win[3][q]);
        }
        if (ebits) atomicOr(&a.err[scene], ebits);
        __syncthreads();
    }
}

// ---------------------------------------------------- PB-MPM cycle G2P
//
// G2P of a PB-MPM cycle (Sec. III-C): positions and F stay fixed during the
// cycles, so each particle's v = sum W v_I and APIC C = 4/dx^2 sum W v_I
// (x_I - x_p)^T are written back in place (storage order), where the next
// cycle's P2G reads them through the same permutation.

constexpr int kVcThreads = 128;

__global__ void __launch_bounds__(kVcThreads) k_g2p_vc(StepArgs a)
{
    __shared__ __align__(128) float4 vw[2][8 * 64];
    __shared__ __align__(16) float4 lin[kWinNodes];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_item[2];
    const int tid = threadIdx.x;
    const int n_act = a.sb.counters[CTR_N_ACT];
    const int cap = a.cap;
    int* work = &a.sb.counters[CTR_WORK_G2P];
    walker_init<kVcThreads>(a, n_act, vw, bar, s_item, work);
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    for (;;) {
        const int item = s_item[buf];
        if (item >= n_act) break;
        if (!walker_next(a, n_act, vw, bar, s_item, work, buf, phase, item)) break;
        const int start = a.sb.act_start[item], count = a.sb.act_count[item];
        const SceneDev sc = a.scenes[a.sb.act_scene[item]];
        const int n = sc.n, nb = sc.nb, lb = a.sb.act_brick[item] - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float c4 = 4.0f * (float)n;
        linearize_window<kVcThreads>(vw[buf], lin);
        __syncthreads();
        for (int k = tid; k < count; k += kVcThreads) {
            const int p = a.sb.perm[start + k];
            int bc[3];
            float f[3], w[9];
            particle_weights(a.in.x[p], a.in.x[cap + p], a.in.x[2 * cap + p], n, bc, f, w);
            const int l0 = min(max(bc[0] - ox, 0), 3), l1 = min(max(bc[1] - oy, 0), 3), l2 = min(max(bc[2] - oz, 0), 3);
            float vv[3] = {0.f, 0.f, 0.f}, B[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) {
                        const float W = w[i] * w[3 + j] * w[6 + kk];
                        const float4 g = lin[(l0 + i) * 36 + (l1 + j) * 6 + (l2 + kk)];
                        const float d0 = (float)i - f[0], d1 = (float)j - f[1], d2 = (float)kk - f[2];
                        const float gv[3] = {g.x, g.y, g.z};
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            vv[r] += W * gv[r];
                            B[3 * r] += W * gv[r] * d0;
                            B[3 * r + 1] += W * gv[r] * d1;
                            B[3 * r + 2] += W * gv[r] * d2;
                        }
                    }
#pragma unroll
            for (int r = 0; r < 3; ++r) a.in.v[(size_t)r * cap + p] = vv[r];
#pragma unroll
            for (int q = 0; q < 9; ++q) a.in.C[(size_t)q * cap + p] = c4 * B[q];
        }
        __syncthreads();
        buf ^= 1;
    }
}

// ------------------------------------------------------- state I/O kernels

__global__ void k_gather_field(PState st, int cap, int p0, int np, int field, void* dst)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np) return;
    const int s = p0 + g;
    const int id = st.id[s];
    if (field == 4) { static_cast<int*>(dst)[g] = id; return; }
    const float* src = field == 0 ? st.x : field == 1 ? st.v : field == 2 ? st.C : st.F;
    const int comps = field < 2 ? 3 : 9;
    float* out = static_cast<float*>(dst) + (size_t)id * comps;
    for (int c = 0; c < comps; ++c) out[c] = src[(size_t)c * cap + s];
}

__global__ void k_scatter_field(PState st, int cap, int p0, int np, int field, const float* src)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np) return;
    const int s = p0 + g;
    const int id = st.id[s];
    float* dst = field == 0 ? st.x : field == 1 ? st.v : field == 2 ? st.C : st.F;
    const int comps = field < 2 ? 3 : 9;
    const float* in = src + (size_t)id * comps;
    for (int c = 0; c < comps; ++c) dst[(size_t)c * cap + s] = in[c];
}

// Inverse of a scene's slot -> id map: inv[id] = slot.
__global__ void k_id_inverse(PState st, int p0, int np, int* inv)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np) return;
    const int id = st.id[p0 + g];
    if ((unsigned)id < (unsigned)np) inv[id] = p0 + g;
}

// State fields <-> host-mapped arrays (pinned host memory the kernel reads or
// writes directly over the host link), in particle-id order: a CTA takes the
// kIoBlock consecutive ids of one contiguous chunk of each host array, so the
// host side moves as whole 16-byte words; the slot side (device memory) is the
// scattered one.  Fields pass one at a time through shared memory.
constexpr int kIoBlock = 128;

template <bool TO_HOST>
__global__ void __launch_bounds__(kIoBlock) k_fields_host(PState st, int cap, int p0, int np,
                                                          const int* __restrict__ inv, HostFields h)
{
    __shared__ __align__(16) float buf[9 * kIoBlock];
    const int t = threadIdx.x;
    const int g0 = blockIdx.x * kIoBlock;
    const int cnt = min(kIoBlock, np - g0);
    // the slot of id g0 + t (ids are a permutation of the scene's slots)
    const int s = t < cnt ? inv[g0 + t] : p0;
    const bool own = t < cnt && (unsigned)(s - p0) < (unsigned)np;
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        float* hp = h.f[f];
        if (!hp) continue;
        const int k = f < 2 ? 3 : 9;
        float* soa = f == 0 ? st.x : f == 1 ? st.v : f == 2 ? st.C : st.F;
        float* chunk = hp + (size_t)g0 * k;
        const int nflt = cnt * k;
        const bool vec = cnt == kIoBlock && (reinterpret_cast<uintptr_t>(chunk) & 15u) == 0;
        if (TO_HOST) {
            if (own)
                for (int c = 0; c < k; ++c) buf[t * k + c] = soa[(size_t)c * cap + s];
            __syncthreads();
            if (vec) {
                for (int i = t; i < nflt / 4; i += kIoBlock)
                    reinterpret_cast<float4*>(chunk)[i] = reinterpret_cast<const float4*>(buf)[i];
            } else {
                for (int i = t; i < nflt; i += kIoBlock) chunk[i] = buf[i];
            }
        } else {
            if (vec) {
                for (int i = t; i < nflt / 4; i += kIoBlock)
                    reinterpret_cast<float4*>(buf)[i] = reinterpret_cast<const float4*>(chunk)[i];
            } else {
                for (int i = t; i < nflt; i += kIoBlock) buf[i] = chunk[i];
            }
            __syncthreads();
            if (own)
                for (int c = 0; c < k; ++c) soa[(size_t)c * cap + s] = buf[t * k + c];
        }
        __syncthreads();  // buf is the next field's
    }
}

__global__ void k_init_particles(PState st, int cap, int p_at, int n, int id0, const float* x, const float* v,
                                 const float* E, const float* nu, float E0, float nu0)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int s = p_at + g;
    for (int d = 0; d < 3; ++d) {
        st.x[(size_t)d * cap + s] = x[3 * (size_t)g + d];
        st.v[(size_t)d * cap + s] = v ? v[3 * (size_t)g + d] : 0.f;
    }
    for (int i = 0; i < 9; ++i) {
        st.C[(size_t)i * cap + s] = 0.f;
        st.F[(size_t)i * cap + s] = (i % 4 == 0) ? 1.f : 0.f;
    }
    const float e = E ? E[g] : E0, q = nu ? nu[g] : nu0;
    st.mu[s] = e / (2.f * (1.f + q));
    st.lam[s] = e * q / ((1.f + q) * (1.f - 2.f * q));
    st.id[s] = id0 + g;
}

__global__ void k_read_grid(const float4* V, const int* brick_epoch, const int* epoch, int scene, int n,
                            int brick_base, float* dst)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)n * n * n;
    if (g >= total) return;
    const int nb = n / 4;
    const int brick = (int)(g >> 6), loc = (int)(g & 63);
    const int B = brick_base + brick;
    if (brick_epoch[B] != epoch[scene] - 1) return;
    const int bx = brick / (nb * nb), by = (brick / nb) % nb, bz = brick % nb;
    const int gi = bx * 4 + (loc >> 4), gj = by * 4 + ((loc >> 2) & 3), gk = bz * 4 + (loc & 3);
    const float4 v = V[(size_t)B * 64 + loc];
    float* o = dst + (((size_t)gi * n + gj) * n + gk) * 4;
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

// ------------------------------------------------------------- launchers

static int n_blocks(long long n, int t) { return (int)((n + t - 1) / t); }

cudaError_t launch_prepare(const StepArgs& a, const PState& st, cudaStream_t s)
{
    if (a.r.np == 0) return cudaSuccess;
    k_prepare<<<n_blocks(a.r.np, 256), 256, 0, s>>>(a, st);
    return cudaGetLastError();
}

cudaError_t launch_sort(const StepArgs& a, cudaStream_t s, bool write_perm)
{
    k_scan<<<a.r.nt, kScanThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int work = a.r.np > a.r.nt ? a.r.np : a.r.nt;
    k_scatter<<<n_blocks(work, 256 * kScatterPer), 256, 0, s>>>(a, write_perm ? 1 : 0);
    return cudaGetLastError();
}

template <int PER>
static constexpr size_t p2g_dyn_smem() { return sizeof(float) * kItemRecFields * P2GShape<PER>::slots; }

cudaError_t prepare_p2g()
{
    cudaError_t e = cudaFuncSetAttribute(k_p2g<2, kP2GStress>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p2g_dyn_smem<2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2g<3, kP2GStress>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p2g_dyn_smem<3>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2g<4, kP2GStress>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p2g_dyn_smem<4>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2g<4, kP2GConstraint>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p2g_dyn_smem<4>());
    return e;
}

cudaError_t launch_p2g(const StepArgs& a, cudaStream_t s)
{
    if (a.solver == MPM_SOLVER_PB) {
        k_p2g<4, kP2GConstraint><<<a.p2g_ctas, kP2GThreads, p2g_dyn_smem<4>(), s>>>(a);
        return cudaGetLastError();
    }
    switch (a.p2g_chunk) {
    case 2 * kP2GThreads: k_p2g<2, kP2GStress><<<a.p2g_ctas, kP2GThreads, p2g_dyn_smem<2>(), s>>>(a); break;
    case 4 * kP2GThreads: k_p2g<4, kP2GStress><<<a.p2g_ctas, kP2GThreads, p2g_dyn_smem<4>(), s>>>(a); break;
    default: k_p2g<3, kP2GStress><<<a.p2g_ctas, kP2GThreads, p2g_dyn_smem<3>(), s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_p2g_std(const StepArgs& a, cudaStream_t s)
{
    k_p2g_std<<<a.p2g_ctas, kStdThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_g2p_vc(const StepArgs& a, cudaStream_t s)
{
    k_g2p_vc<<<a.persistent_ctas, kVcThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int occupancy_p2g_std()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_p2g_std, kStdThreads, 0);
    return b;
}

cudaError_t launch_grid(const StepArgs& a, cudaStream_t s)
{
    if (!a.any_rigid) k_grid_plain<<<a.grid_plain_ctas, kGridThreads, 0, s>>>(a);
    else if (a.rigid_ext) k_grid<true><<<a.grid_ctas, kGridThreads, 0, s>>>(a);
    else k_grid<false><<<a.grid_ctas, kGridThreads, 0, s>>>(a);
    k_grid_clear<<<a.grid_plain_ctas, kGridThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int FLAGS>
static void launch_g2p_variant(const StepArgs& a, cudaStream_t s)
{
    const int c = a.persistent_ctas;
    if (a.g2p_regs64) {
        switch (a.g2p_threads) {
        case 128: k_g2p<128, 8, FLAGS><<<c, 128, 0, s>>>(a); break;
        case 512: k_g2p<512, 2, FLAGS><<<c, 512, 0, s>>>(a); break;
        default: k_g2p<256, 4, FLAGS><<<c, 256, 0, s>>>(a); break;
        }
    } else {
        switch (a.g2p_threads) {
        case 128: k_g2p<128, 7, FLAGS><<<c, 128, 0, s>>>(a); break;
        case 512: k_g2p<512, 1, FLAGS><<<c, 512, 0, s>>>(a); break;
        default: k_g2p<256, 3, FLAGS><<<c, 256, 0, s>>>(a); break;
        }
    }
}

// The standard-MPM and PB-MPM variants exist in one launch shape only (128
// threads, 64 registers): the MLS-MPM shapes are what the tuner explores.
cudaError_t launch_g2p(const StepArgs& a, cudaStream_t s)
{
    const int c = a.persistent_ctas;
    // the push-out variant only where a scene has a solid shape: blades, needles and
    // segments push nothing out
    if (a.solver == MPM_SOLVER_STANDARD) {
        if (a.any_solid) k_g2p<128, 8, kG2PStdGrad | kG2PSolids><<<c, 128, 0, s>>>(a);
        else k_g2p<128, 8, kG2PStdGrad><<<c, 128, 0, s>>>(a);
    } else if (a.solver == MPM_SOLVER_PB) {
        if (a.any_solid) k_g2p<128, 8, kG2PNoStress | kG2PSolids><<<c, 128, 0, s>>>(a);
        else k_g2p<128, 8, kG2PNoStress><<<c, 128, 0, s>>>(a);
    } else if (a.any_solid) {
        launch_g2p_variant<kG2PSolids>(a, s);
    } else {
        launch_g2p_variant<0>(a, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_g2p2g(const StepArgs& a, cudaStream_t s)
{
    k_g2p2g<<<a.fused_ctas, kFusedThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int occupancy_grid()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_grid<true>, kGridThreads, 0);
    return b;
}

int occupancy_grid_plain()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_grid_plain, kGridThreads, 0);
    return b;
}

int occupancy_g2p2g()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p2g, kFusedThreads, 0);
    return b;
}

cudaError_t launch_gather_field(const PState& st, int cap, int p0, int np, int field, void* dst, cudaStream_t s)
{
    if (np == 0) return cudaSuccess;
    k_gather_field<<<n_blocks(np, 256), 256, 0, s>>>(st, cap, p0, np, field, dst);
    return cudaGetLastError();
}

cudaError_t launch_id_inverse(const PState& st, int p0, int np, int* inv, cudaStream_t s)
{
    if (np == 0) return cudaSuccess;
    k_id_inverse<<<n_blocks(np, 256), 256, 0, s>>>(st, p0, np, inv);
    return cudaGetLastError();
}

cudaError_t launch_fields_host(const PState& st, int cap, int p0, int np, const int* inv, const HostFields& h,
                               bool to_host, cudaStream_t s)
{
    if (np == 0) return cudaSuccess;
    if (to_host) k_fields_host<true><<<n_blocks(np, kIoBlock), kIoBlock, 0, s>>>(st, cap, p0, np, inv, h);
    else k_fields_host<false><<<n_blocks(np, kIoBlock), kIoBlock, 0, s>>>(st, cap, p0, np, inv, h);
    return cudaGetLastError();
}

cudaError_t launch_scatter_field(const PState& st, int cap, int p0, int np, int field, const float* src, cudaStream_t s)
{
    if (np == 0) return cudaSuccess;
    k_scatter_field<<<n_blocks(np, 256), 256, 0, s>>>(st, cap, p0, np, field, src);
    return cudaGetLastError();
}

cudaError_t launch_init_particles(const PState& st, int cap, int p_at, int n, int id0, const float* x, const float* v,
                                  const float* E, const float* nu, float E0, float nu0, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_init_particles<<<n_blocks(n, 256), 256, 0, s>>>(st, cap, p_at, n, id0, x, v, E, nu, E0, nu0);
    return cudaGetLastError();
}

cudaError_t launch_read_grid(const float4* V, const int* brick_epoch, const int* epoch, const SceneDev*, int scene,
                             int n, int brick_base, float* dst, cudaStream_t s)
{
    const long long total = (long long)n * n * n;
    k_read_grid<<<n_blocks(total, 256), 256, 0, s>>>(V, brick_epoch, epoch, scene, n, brick_base, dst);
    return cudaGetLastError();
}

int occupancy_p2g(int chunk)
{
    int b = 0;
    if (chunk == 2 * kP2GThreads)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_p2g<2, kP2GStress>, kP2GThreads, p2g_dyn_smem<2>());
    else if (chunk == 4 * kP2GThreads)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_p2g<4, kP2GStress>, kP2GThreads, p2g_dyn_smem<4>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_p2g<3, kP2GStress>, kP2GThreads, p2g_dyn_smem<3>());
    return b;
}

int occupancy_g2p(int threads, int regs64)
{
    // the variant with the push-out uses the same registers and a little more
    // shared memory; its occupancy bounds both
    int b = 0;
    if (regs64) {
        if (threads == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<128, 8, kG2PSolids>, 128, 0);
        else if (threads == 512) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<512, 2, kG2PSolids>, 512, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<256, 4, kG2PSolids>, 256, 0);
    } else {
        if (threads == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<128, 7, kG2PSolids>, 128, 0);
        else if (threads == 512) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<512, 1, kG2PSolids>, 512, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_g2p<256, 3, kG2PSolids>, 256, 0);
    }
    return b;
}

}  // namespace mpm
