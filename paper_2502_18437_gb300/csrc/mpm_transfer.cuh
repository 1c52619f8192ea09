// Device helpers shared by the forward and adjoint transfer kernels: PTX
// wrappers (mbarrier, bulk-copy TMA, vector reductions), brick keys and ranks,
// B-spline weights, P2G coefficients, the P2G item schedule and accumulation,
// halo staging.
#pragma once

#include "mpm_kernels.cuh"

namespace mpm {

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_add_v4(float4* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------- brick key + rank

// Sort key of a particle: its brick (global index) x 64 + its base cell inside
// the brick.  The sort orders by brick (key >> 6); P2G reads the cell back.
__device__ __forceinline__ int cell_key(const SceneDev& sc, float x0, float x1, float x2, unsigned& ood)
{
    int c0, c1, c2;
    ood |= (unsigned)(base_cell(x0, sc.n, c0) | base_cell(x1, sc.n, c1) | base_cell(x2, sc.n, c2));
    const int brick = sc.brick_base + ((c0 >> 2) * sc.nb + (c1 >> 2)) * sc.nb + (c2 >> 2);
    return brick * 64 + ((c0 & 3) * 16 + (c1 & 3) * 4 + (c2 & 3));
}

// Warp-aggregated rank: lanes with the same brick get consecutive ranks from
// one atomic (all 32 lanes call it; `valid` marks lanes with a particle).  It
// also keeps the scan's bookkeeping of the next substep:
//  - the brick's particle count (the rank base) and its scan tile's sums;
//  - for the first warp to add particles to a brick, the brick and its 7 upper
//    neighbours (+1 in any subset of the axes) are flagged as node bricks the
//    scan must activate (a particle's 3-node stencil reaches at most 2 nodes
//    past its base cell, i.e. into the next brick).  Each flag is set with an
//    exchange, so that its tile counts every node brick exactly once.
// brick is the global brick index of the key.  add_x = false leaves the tile's
// particle count to the caller (which then aggregates it itself).
__device__ __forceinline__ int aggregated_rank_mark(const SortBufs& sb, const SceneDev& sc, int brick, bool valid,
                                                    bool add_x = true)
{
    const unsigned active = __ballot_sync(kFull, valid);
    int rank = 0;
    const unsigned peers = __match_any_sync(kFull, valid ? brick : -1) & active;
    if (valid) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) {
            const int np = __popc(peers);
            const int lb = brick - sc.brick_base;
            int4* ts = sb.tile_sum + sc.tile_base;
            base = atomicAdd(&sb.cnt[brick], np);
            if (add_x) atomicAdd(&ts[lb >> sb.tile_shift].x, np);
            if (base < kBigBrick && base + np >= kBigBrick) atomicAdd(&ts[lb >> sb.tile_shift].w, 1);
            if (base == 0) {
                atomicAdd(&ts[lb >> sb.tile_shift].y, 1);
                const int nb = sc.nb;
                int bx, by, bz;
                brick_coords(nb, sc.nb_log2, lb, bx, by, bz);
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int ex = bx + (o >> 2), ey = by + ((o >> 1) & 1), ez = bz + (o & 1);
                    if (ex < nb && ey < nb && ez < nb) {
                        const int ln = (ex * nb + ey) * nb + ez;
                        if (atomicExch(&sb.nflag[sc.brick_base + ln], 1) == 0) atomicAdd(&ts[ln >> sb.tile_shift].z, 1);
                    }
                }
            }
        }
        base = __shfl_sync(peers, base, leader);
        rank = base + __popc(peers & ((1u << lane) - 1u));
    }
    return rank;
}

// ------------------------------------------------------ transfer helpers

constexpr int kRecFields = 21;  // w0[3] w1[3] w2[3] q[3] Ad[9]

// Base cells, fractional offsets and quadratic B-spline weights of a position.
__device__ __forceinline__ unsigned particle_weights(float x0, float x1, float x2, int n, int b[3], float f[3],
                                                     float w[9])
{
    const float fn = (float)n;
    const unsigned ood = base_cell(x0, n, b[0]) | base_cell(x1, n, b[1]) | base_cell(x2, n, b[2]);
    f[0] = __fmaf_rn(x0, fn, -(float)b[0]);
    f[1] = __fmaf_rn(x1, fn, -(float)b[1]);
    f[2] = __fmaf_rn(x2, fn, -(float)b[2]);
    bspline(f[0], w);
    bspline(f[1], w + 3);
    bspline(f[2], w + 6);
    return ood ? MPM_EBIT_OUT_OF_DOMAIN : 0u;
}

// P2G coefficients (Eq. 8 with the APIC particle momentum, M^-1 = 4/dx^2 of
// Eq. 7, V sigma = V0 tau): the momentum a particle gives node (i,j,k) of its
// stencil is W_ijk (q + Ad (i,j,k)) with Ad = (m C - dt V0 M^-1 tau) dx and
// q = m v - Ad f, so that Ad ((i,j,k) - f) = A (x_I - x_p).
__device__ __forceinline__ void p2g_coeffs(float m, float kA, float dxs, const float v[3], const float C[9],
                                           const float t6[6], const float f[3], float q[3], float Ad[9])
{
    const float tau[9] = {t6[0], t6[1], t6[2], t6[1], t6[3], t6[4], t6[2], t6[4], t6[5]};
#pragma unroll
    for (int i = 0; i < 9; ++i) Ad[i] = (m * C[i] - kA * tau[i]) * dxs;
#pragma unroll
    for (int r = 0; r < 3; ++r) q[r] = m * v[r] - (Ad[3 * r] * f[0] + Ad[3 * r + 1] * f[1] + Ad[3 * r + 2] * f[2]);
}

template <int N>
__device__ __forceinline__ void put_record(float (*rec)[N], int k, const float w[9], const float q[3], const float Ad[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[i][k] = w[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) rec[9 + i][k] = q[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[12 + i][k] = Ad[i];
}

// Phase B of the per-cell accumulation: thread (cell, slice) adds the
// contributions of the particles of its cell (order[beg..end)) to the 9 nodes
// cell + (slice, j, k) in registers.
template <int N>
__device__ __forceinline__ void cell_accumulate(const float (*rec)[N], const short* order, int beg, int end, int slice,
                                                float acc_w[9], float acc_p[9][3])
{
    const float si = (float)slice;
    for (int j = beg; j < end; ++j) {
        const int k = order[j];
        const float wi = rec[slice][k];
        const float wy[3] = {rec[3][k], rec[4][k], rec[5][k]};
        const float wz[3] = {rec[6][k], rec[7][k], rec[8][k]};
        // r(j,k) = q + Ad (slice, j, k)
        const float r0 = rec[9][k] + si * rec[12][k], r1 = rec[10][k] + si * rec[15][k], r2 = rec[11][k] + si * rec[18][k];
        const float a01 = rec[13][k], a11 = rec[16][k], a21 = rec[19][k];
        const float a02 = rec[14][k], a12 = rec[17][k], a22 = rec[20][k];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const float wij = wi * wy[jj];
            const float s0 = r0 + a01 * jj, s1 = r1 + a11 * jj, s2 = r2 + a21 * jj;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const float W = wij * wz[kk];
                const int q = jj * 3 + kk;
                acc_w[q] += W;
                acc_p[q][0] += W * (s0 + a02 * kk);
                acc_p[q][1] += W * (s1 + a12 * kk);
                acc_p[q][2] += W * (s2 + a22 * kk);
            }
        }
    }
}

// Exclusive scan of the 64 per-cell counts by warp 0.
__device__ __forceinline__ void scan_cells(const int* cell_cnt, int* cell_off, int tid)
{
    if (tid < 32) {
        const int c_a = cell_cnt[2 * tid], c_b = cell_cnt[2 * tid + 1];
        int incl = c_a + c_b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, d);
            if (tid >= d) incl += t;
        }
        const int excl = incl - c_a - c_b;
        cell_off[2 * tid] = excl;
        cell_off[2 * tid + 1] = excl + c_a;
        if (tid == 31) cell_off[64] = incl;
    }
}

// floor(y / L) for 0 <= y < 2^22 from one single-precision product with
// inv = 1/L: the exact quotient (y + 0.5)/L lies at least 0.5/L away from an
// integer, which bounds the rounding error of the product from above.
__device__ __forceinline__ int div_small(int y, float inv) { return (int)(((float)y + 0.5f) * inv); }

// Work items of one P2G pass.  The particles of each cell (contiguous in the
// cell-sorted order) are cut into items of at most L particles, L being the
// smallest length that gives at most 64 items; items of length L come first,
// then the shorter remainders, longest first (eight length classes), so that
// the 32 lanes of a warp run loops of nearly the same length.  Called by warp
// 0 once cell_cnt holds the pass's per-cell counts (cn <= 4095 particles);
// writes cell_off (exclusive scan of cell_cnt, 65 entries), the item table
// (cell, first position in the cell-sorted order, length), the item count, L,
// per cell the index of its first full item, its number of full items and the
// index of its remainder item (-1: none), and s_len = {L, longest item among
// items 0..31, longest among items 32..63}.
__device__ __forceinline__ void build_items(const int* cell_cnt, int* cell_off, int cn, short* it_cell, short* it_beg,
                                            short* it_len, int* n_items, short* c_full, short* c_nf, short* c_rem,
                                            int* s_len)
{
    const int lane = threadIdx.x & 31;
    const int ca = 2 * lane, cb = ca + 1;
    const int ka = cell_cnt[ca], kb = cell_cnt[cb];
    const int kmax = __reduce_max_sync(kFull, max(ka, kb));
    // smallest L in [L0, max(L0, kmax)] with sum_c ceil(k_c / L) <= 64 (the upper
    // end always qualifies: every cell is then one item at most)
    int lo = max(1, (cn + 63) >> 6), hi = max(lo, kmax);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float inv = 1.0f / (float)mid;
        const int items =
            __reduce_add_sync(kFull, div_small(ka + mid - 1, inv) + div_small(kb + mid - 1, inv));
        if (items <= 64) hi = mid;
        else lo = mid + 1;
    }
    const int L = lo;
    const float inv = 1.0f / (float)L;
    const int nfa = div_small(ka, inv), nfb = div_small(kb, inv);
    const int ra = ka - nfa * L, rb = kb - nfb * L;
    // one scan of (count, full items) packed in 16-bit halves
    const int own = (ka + kb) | ((nfa + nfb) << 16);
    int incl = own;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
    }
    const int excl = incl - own;
    const int offa = excl & 0xffff, offb = offa + ka;
    const int fa = excl >> 16, fb = fa + nfa;
    const int n_full = __shfl_sync(kFull, incl, 31) >> 16;
    cell_off[ca] = offa;
    cell_off[cb] = offb;
    if (lane == 31) cell_off[64] = incl & 0xffff;
    // remainders in eight length classes, longest class first, cell order inside
    const int ga = ra > 0 ? div_small(8 * (L - ra), inv) : 8, gb = rb > 0 ? div_small(8 * (L - rb), inv) : 8;
    const unsigned lt = (1u << lane) - 1u;
    int pa = -1, pb = -1, base = n_full;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const unsigned ma = __ballot_sync(kFull, ga == g), mb = __ballot_sync(kFull, gb == g);
        if (ga == g) pa = base + __popc(ma & lt) + __popc(mb & lt);
        if (gb == g) pb = base + __popc(ma & (lt | (1u << lane))) + __popc(mb & lt);
        base += __popc(ma) + __popc(mb);
    }
    for (int j = 0; j < nfa; ++j) {
        it_cell[fa + j] = (short)ca;
        it_beg[fa + j] = (short)(offa + j * L);
        it_len[fa + j] = (short)L;
    }
    for (int j = 0; j < nfb; ++j) {
        it_cell[fb + j] = (short)cb;
        it_beg[fb + j] = (short)(offb + j * L);
        it_len[fb + j] = (short)L;
    }
    if (pa >= 0) {
        it_cell[pa] = (short)ca;
        it_beg[pa] = (short)(offa + nfa * L);
        it_len[pa] = (short)ra;
    }
    if (pb >= 0) {
        it_cell[pb] = (short)cb;
        it_beg[pb] = (short)(offb + nfb * L);
        it_len[pb] = (short)rb;
    }
    c_full[ca] = (short)fa;
    c_full[cb] = (short)fb;
    c_nf[ca] = (short)nfa;
    c_nf[cb] = (short)nfb;
    c_rem[ca] = (short)pa;
    c_rem[cb] = (short)pb;
    __syncwarp();
    // longest item of each group of 32 (the record rows of that warp)
    const int r0 = __reduce_max_sync(kFull, lane < base ? (int)it_len[lane] : 0);
    const int r1 = __reduce_max_sync(kFull, lane + 32 < base ? (int)it_len[lane + 32] : 0);
    if (lane == 31) {
        *n_items = base;
        s_len[0] = L;
        s_len[1] = r0;
        s_len[2] = r1;
    }
}

// Record of one particle for the item schedule: fractional offsets f (3),
// q (3) and Ad (9) of p2g_coeffs; the weights are recomputed in phase B.
constexpr int kItemRecFields = 15;

template <int N>
__device__ __forceinline__ void put_item_record(float (*rec)[N], int k, const float f[3], const float q[3],
                                                const float Ad[9])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) rec[i][k] = f[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) rec[3 + i][k] = q[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[6 + i][k] = Ad[i];
}

// Phase B of the item schedule: thread (item, slice) adds the contributions of
// the item's particles, whose records sit at slots slot0, slot0 + stride, ...,
// to the 9 nodes cell + (slice, j, k) in registers.  The weights follow the
// quadratic B-spline of bspline(): slice i needs w_i(f_x) only, written as
// alpha + beta (f - gamma)^2.  The sums are kept in pairs, (p_x, p_y) in
// acc_a and (p_z, weight) in acc_b, each updated by one paired FMA.
template <int N>
__device__ __forceinline__ void item_accumulate(const float (*rec)[N], int slot0, int stride, int len, int slice,
                                                float2 acc_a[9], float2 acc_b[9])
{
    const float si = (float)slice;
    const float gam = slice == 0 ? 1.5f : (slice == 1 ? 1.0f : 0.5f);
    const float bet = slice == 1 ? -1.0f : 0.5f, alp = slice == 1 ? 0.75f : 0.0f;
    int k = slot0;
    for (int j = 0; j < len; ++j, k += stride) {
        const float fx = rec[0][k], fy = rec[1][k], fz = rec[2][k];
        const float dxw = fx - gam;
        const float wi = __fmaf_rn(bet * dxw, dxw, alp);
        float wy[3], wz[3];
        bspline(fy, wy);
        bspline(fz, wz);
        // value of node (slice, jj, kk): r + a1 jj + a2 kk (r includes the slice's term)
        const float2 r01 = make_float2(__fmaf_rn(si, rec[6][k], rec[3][k]), __fmaf_rn(si, rec[9][k], rec[4][k]));
        const float r2 = __fmaf_rn(si, rec[12][k], rec[5][k]);
        const float2 a1 = make_float2(rec[7][k], rec[10][k]), a2 = make_float2(rec[8][k], rec[11][k]);
        const float a21 = rec[13][k], a22 = rec[14][k];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const float wij = wi * wy[jj];
            const float fj = (float)jj;
            const float2 s01 = jj == 0 ? r01 : __ffma2_rn(make_float2(fj, fj), a1, r01);
            const float s2 = __fmaf_rn(a21, fj, r2);
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const float W = wij * wz[kk];
                const float fk = (float)kk;
                const int q = jj * 3 + kk;
                const float2 v01 = kk == 0 ? s01 : __ffma2_rn(make_float2(fk, fk), a2, s01);
                const float2 v2w = make_float2(__fmaf_rn(a22, fk, s2), 1.0f);
                acc_a[q] = __ffma2_rn(make_float2(W, W), v01, acc_a[q]);
                acc_b[q] = __ffma2_rn(make_float2(W, W), v2w, acc_b[q]);
            }
        }
    }
}

// Global node index of node (gi, gj, gk) of a scene (brick layout).
__device__ __forceinline__ int node_index(const SceneDev& sc, int gi, int gj, int gk)
{
    const int brick = sc.brick_base + ((gi >> 2) * sc.nb + (gj >> 2)) * sc.nb + (gk >> 2);
    return brick * 64 + (gi & 3) * 16 + (gj & 3) * 4 + (gk & 3);
}

__device__ __forceinline__ void issue_halo(const StepArgs& a, int item, float4* dst, unsigned long long* bar)
{
    const int b = a.sb.act_brick[item];
    const SceneDev& sc = a.scenes[a.sb.act_scene[item]];
    const int nb = sc.nb, lb = b - sc.brick_base;
    int bx, by, bz;
    brick_coords(nb, sc.nb_log2, lb, bx, by, bz);
    fence_proxy_async();
    unsigned bytes = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o)
        if (bx + (o >> 2) < nb && by + ((o >> 1) & 1) < nb && bz + (o & 1) < nb) bytes += 64 * sizeof(float4);
    mbar_expect_tx(bar, bytes);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int ex = bx + (o >> 2), ey = by + ((o >> 1) & 1), ez = bz + (o & 1);
        if (ex < nb && ey < nb && ez < nb)
            bulk_g2s(dst + o * 64, &a.V[(sc.brick_base + (ex * nb + ey) * nb + ez) * 64], 64 * sizeof(float4), bar);
    }
}

// Shared prologue of the brick-walking kernels: mbarriers, first halo.
template <int BLOCK>
__device__ __forceinline__ void walker_init(const StepArgs& a, int n_act, float4 (*vw)[8 * 64], unsigned long long* bar,
                                            int* s_item, int* work)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        const int first = atomicAdd(work, 1);
        s_item[0] = first;
        if (first < n_act) issue_halo(a, first, vw[0], &bar[0]);
    }
    __syncthreads();
}

// Epilogue of the forward G2P launches, run by every CTA on its way out: the
// last CTA to finish advances the scene clocks and substep counters (read by
// the next grid update and the state readback).  No CTA of the launch reads a
// clock after it has counted itself out, so the clocks stay constant while
// G2P evaluates rigid poses at the end of the substep.
__device__ __forceinline__ void walker_exit(const StepArgs& a)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&a.sb.counters[CTR_DONE_G2P], 1);
        if (done == (int)gridDim.x - 1) {
            __threadfence();
            for (int s = a.r.s0; s < a.r.s1; ++s) {
                a.t_scene[s] += (double)a.dt;
                a.epoch[s] += 1;
            }
            a.sb.counters[CTR_DONE_G2P] = 0;
        }
    }
}

// Poses at the end of the substep (clock + dt) of the solid rigids of a scene,
// staged in shared memory by the threads tid < kMaxRigids; returns the rigid
// slots in use (shapes other than sphere and box are staged with type -1).
__device__ __forceinline__ void rigid_pose_at(const RigidDev& src, double t_now, float c[3], float R[9])
{
    const float tau = (float)(t_now - src.t_set);
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = src.c0[i] + tau * src.vel[i];
    // q(tau) = exp(tau omega / 2) * q0
    const float wx = src.omega[0], wy = src.omega[1], wz = src.omega[2];
    const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
    float qw = src.q0[0], qx = src.q0[1], qy = src.q0[2], qz = src.q0[3];
    if (wn > 0.f) {
        float sh, ch;
        sincosf(0.5f * wn * tau, &sh, &ch);
        const float ax = wx / wn * sh, ay = wy / wn * sh, az = wz / wn * sh;
        const float nw = ch * qw - ax * qx - ay * qy - az * qz;
        const float nx = ch * qx + ax * qw + ay * qz - az * qy;
        const float ny = ch * qy - ax * qz + ay * qw + az * qx;
        const float nz = ch * qz + ax * qy - ay * qx + az * qw;
        qw = nw; qx = nx; qy = ny; qz = nz;
    }
    quat_to_mat(qw, qx, qy, qz, R);
}

__device__ __forceinline__ void stage_solids(const StepArgs& a, int scene, SolidPose* poses)
{
    const int tid = threadIdx.x;
    const int nr = a.scenes[scene].n_rigid;
    if (tid < nr) {
        const RigidDev& src = a.rigids[scene * kMaxRigids + tid];
        SolidPose& P = poses[tid];
        P.type = (src.type == MPM_SPHERE || src.type == MPM_BOX) ? src.type : -1;
        rigid_pose_at(src, a.t_scene[scene] + (double)a.dt, P.c, P.R);
        P.radius = src.radius;
#pragma unroll
        for (int i = 0; i < 3; ++i) P.half[i] = src.half[i];
    }
}

// Particle push-out (Sec. IV-A): a particle that ends the substep inside a
// solid rigid (sdf < 0 at the rigid's pose at the end of the substep) moves
// to the nearest surface point, x - sdf(x) n(x); rigids in id order.  Blades
// and line segments push nothing out (the tissue closes around them).
__device__ __forceinline__ void push_out(const SolidPose* poses, int nr, float x[3])
{
    for (int r = 0; r < nr; ++r) {
        const SolidPose& P = poses[r];
        if (P.type == MPM_SPHERE) {
            const float d0 = x[0] - P.c[0], d1 = x[1] - P.c[1], d2 = x[2] - P.c[2];
            const float l = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            if (l < P.radius) {
                if (l > 0.f) {
                    const float k = P.radius / l;
                    x[0] = P.c[0] + k * d0;
                    x[1] = P.c[1] + k * d1;
                    x[2] = P.c[2] + k * d2;
                } else {  // at the centre: along the body y axis
                    x[0] = P.c[0] + P.radius * P.R[1];
                    x[1] = P.c[1] + P.radius * P.R[4];
                    x[2] = P.c[2] + P.radius * P.R[7];
                }
            }
        } else if (P.type == MPM_BOX) {
            const float d0 = x[0] - P.c[0], d1 = x[1] - P.c[1], d2 = x[2] - P.c[2];
            float p[3] = {P.R[0] * d0 + P.R[3] * d1 + P.R[6] * d2, P.R[1] * d0 + P.R[4] * d1 + P.R[7] * d2,
                          P.R[2] * d0 + P.R[5] * d1 + P.R[8] * d2};
            const float q0 = fabsf(p[0]) - P.half[0], q1 = fabsf(p[1]) - P.half[1], q2 = fabsf(p[2]) - P.half[2];
            if (q0 < 0.f && q1 < 0.f && q2 < 0.f) {
                // nearest face: the axis of the largest q (ties to the lower axis)
                const int ax = (q0 >= q1 && q0 >= q2) ? 0 : (q1 >= q2 ? 1 : 2);
                p[ax] = p[ax] >= 0.f ? P.half[ax] : -P.half[ax];
                x[0] = P.c[0] + P.R[0] * p[0] + P.R[1] * p[1] + P.R[2] * p[2];
                x[1] = P.c[1] + P.R[3] * p[0] + P.R[4] * p[1] + P.R[5] * p[2];
                x[2] = P.c[2] + P.R[6] * p[0] + P.R[7] * p[1] + P.R[8] * p[2];
            }
        }
    }
}

// Prefetch the next brick's halo and wait for this one; false on timeout (the
// CTA must then return).
__device__ __forceinline__ bool walker_next(const StepArgs& a, int n_act, float4 (*vw)[8 * 64], unsigned long long* bar,
                                            int* s_item, int* work, int buf, unsigned* phase, int item)
{
    if (threadIdx.x == 0) {
        const int next = atomicAdd(work, 1);
        s_item[buf ^ 1] = next;
        if (next < n_act) issue_halo(a, next, vw[buf ^ 1], &bar[buf ^ 1]);
    }
    const bool ok = mbar_wait_bounded(&bar[buf], phase[buf]);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(&a.err[a.sb.act_scene[item]], MPM_EBIT_TIMEOUT);
        mbar_wait_bounded(&bar[buf], phase[buf]);  // let copies in flight land before leaving
        mbar_wait_bounded(&bar[buf ^ 1], phase[buf ^ 1]);
        return false;
    }
    phase[buf] ^= 1u;
    return true;
}

}  // namespace mpm
