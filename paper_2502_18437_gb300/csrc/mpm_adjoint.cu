// Reverse-mode gradients of the MLS-MPM substep (hand-written adjoint
// kernels) and the tape that records a trajectory for them.
//
// One substep (Algorithm 1 of arXiv 2502.18437, walls as projections, no
// rigid contact, no plasticity) maps the particle state s_k = (x, v, C, F) to
// s_{k+1}.  Its reverse, given the adjoint of s_{k+1}:
//  G2P^-1: F' = (I + dt C') F, x' = x + dt v', v' = sum W v_I,
//          C' = 4n sum W v_I (o - f)^T  (o the node offset, f = x/dx - base)
//          -> F_bar = (I + dt C')^T F'_bar,  Ct = C'_bar + dt F'_bar F^T,
//             vt = v'_bar + dt x'_bar,  v_I_bar += W (vt + 4n Ct (o - f)),
//             x_bar = x'_bar + sum grad W (v_I.vt + 4n v_I.Ct(o - f))
//                    - 4n^2 sum W Ct^T v_I   (the f in (o - f))
//  grid^-1: v_I = wall projection of u_I = P_I / m_I + dt g
//          -> u_bar = masked v_I_bar, P_I_bar = u_bar / m_I,
//             m_I_bar = -u_bar . (u_I - dt g) / m_I
//  P2G^-1: m_I += W m, P_I += W (m v + A d), A = m C - dt V0 (4/dx^2) tau(F),
//          d = x_I - x_p
//          -> v_bar = sum W m P_I_bar, A_bar = sum W P_I_bar d^T,
//             C_bar = m A_bar, tau_bar = -dt V0 (4/dx^2) A_bar,
//             x_bar += sum grad W (m m_I_bar + P_I_bar.(m v + A d)) - sum W A^T P_I_bar,
//             F_bar += d tau/d F ^T tau_bar, (mu, lambda)_bar likewise.
// Stress derivatives: Neo-Hookean in closed form; fixed-corotated through
// the derivative of the polar rotation R of F = R S, which solves the
// Sylvester equation Omega S + S Omega = R^T dF - dF^T R for Omega = R^T dR;
// in the eigenbasis of S the solution is Omega_ij = M_ij / (s_i + s_j).
//
// Tape: mpm_tape_begin checkpoints the state; every recorded substep keeps
// its sort permutation (so that recomputed substeps store particles in the
// same order as the recorded ones) and every K-th state is checkpointed.
// mpm_backward walks the segments backwards: restore the checkpoint,
// recompute the segment's states, then reverse each substep (recompute its
// P2G and grid update, then G2P^-1, grid^-1, P2G^-1).
#include <algorithm>
#include <cstring>
#include <vector>

#include "mpm_ctx.cuh"
#include "mpm_transfer.cuh"

using namespace mpm;

struct mpm_tape {
    int K = 0, max_steps = 0, cap = 0;
    std::vector<float> dts;
    std::vector<float*> ckpt;  // states at substeps 0, K, 2K, ...
    float* seg = nullptr;      // K states of the segment being reversed
    int* perms = nullptr;      // [max_steps][cap] recorded permutations
    float* adj = nullptr;      // 2 adjoint states, [2][24][cap]
    float* gmat = nullptr;     // [2][cap] mu, lambda gradients (global particle order)
    float* io = nullptr;       // [28][cap] staged gradient inputs / outputs
};

namespace mpm {

constexpr int kAdjThreads = 256;

struct AdjState {
    float* x;
    float* v;
    float* C;
    float* F;
};

static AdjState adj_view(float* base, int cap)
{
    AdjState a;
    a.x = base;
    a.v = base + 3 * (size_t)cap;
    a.C = base + 6 * (size_t)cap;
    a.F = base + 15 * (size_t)cap;
    return a;
}

struct AdjArgs {
    StepArgs a;
    AdjState nxt;  // adjoint of s_{k+1}, by slot of substep k's sort
    AdjState cur;  // adjoint of s_k, by storage index of s_k
    float* gmu;    // d L / d mu per particle (global order)
    float* glam;
};

__device__ __forceinline__ int scene_of(const StepArgs& a, int i)
{
    int lo = a.r.s0, hi = a.r.s1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.scenes[mid].p_begin <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Cofactor matrix cof(F) = det(F) F^-T.
__device__ __forceinline__ void cofactor(const float F[9], float K[9])
{
    K[0] = F[4] * F[8] - F[5] * F[7];
    K[1] = F[5] * F[6] - F[3] * F[8];
    K[2] = F[3] * F[7] - F[4] * F[6];
    K[3] = F[2] * F[7] - F[1] * F[8];
    K[4] = F[0] * F[8] - F[2] * F[6];
    K[5] = F[1] * F[6] - F[0] * F[7];
    K[6] = F[1] * F[5] - F[2] * F[4];
    K[7] = F[2] * F[3] - F[0] * F[5];
    K[8] = F[0] * F[4] - F[1] * F[3];
}

// Kirchhoff stress (full 3x3) of F, and the vector-Jacobian product of
// tau(F; mu, lambda) with tau_bar.
__device__ void stress_and_vjp(int model, const float F[9], float mu, float lam, float tau[9], const float* tb,
                               float Fb[9], float& mub, float& lamb)
{
    float K[9];
    cofactor(F, K);
    if (model == MPM_NEO_HOOKEAN) {
        const float J = F[0] * K[0] + F[1] * K[1] + F[2] * K[2];
        const float lnJ = J > 0.f ? logf(J) : 0.f;
        float FFt[9];
        mul_abt(F, F, FFt);
#pragma unroll
        for (int i = 0; i < 9; ++i) tau[i] = mu * (FFt[i] - ((i % 4 == 0) ? 1.f : 0.f)) + ((i % 4 == 0) ? lam * lnJ : 0.f);
        if (!tb) return;
        const float tr = tb[0] + tb[4] + tb[8];
        // F_bar = mu (tb + tb^T) F + lambda tr(tb) F^-T
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) acc += (tb[3 * r + k] + tb[3 * k + r]) * F[3 * k + c];
                Fb[3 * r + c] = mu * acc + (J != 0.f ? lam * tr * K[3 * r + c] / J : 0.f);
            }
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) m += tb[i] * (FFt[i] - ((i % 4 == 0) ? 1.f : 0.f));
        mub = m;
        lamb = tr * lnJ;
        return;
    }
    float U[9], s[3], V[9], R[9], P[9];
    svd3(F, U, s, V);
    mul_abt(U, V, R);
    const float J = s[0] * s[1] * s[2];
#pragma unroll
    for (int i = 0; i < 9; ++i) P[i] = F[i] - R[i];
    float PFt[9];
    mul_abt(P, F, PFt);
#pragma unroll
    for (int i = 0; i < 9; ++i) tau[i] = 2.f * mu * PFt[i] + ((i % 4 == 0) ? lam * (J - 1.f) * J : 0.f);
    if (!tb) return;
    const float tr = tb[0] + tb[4] + tb[8];
    // G = tb F;  F_bar = 2 mu G + 2 mu tb^T P + lambda (2J - 1) tr(tb) J F^-T + polar part
    float G[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            G[3 * r + c] = tb[3 * r] * F[c] + tb[3 * r + 1] * F[3 + c] + tb[3 * r + 2] * F[6 + c];
            Fb[3 * r + c] = 2.f * mu * (G[3 * r + c] + tb[r] * P[c] + tb[3 + r] * P[3 + c] + tb[6 + r] * P[6 + c]) +
                            lam * (2.f * J - 1.f) * tr * K[3 * r + c];
        }
    // polar part: R_bar = -2 mu G; K = R^T R_bar; X = V [ (V^T skew(K) V)_ij / (s_i + s_j) ] V^T; F_bar += 2 R X
    float Kr[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Kr[3 * r + c] = -2.f * mu * (R[r] * G[c] + R[3 + r] * G[3 + c] + R[6 + r] * G[6 + c]);
    float Ks[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Ks[3 * r + c] = 0.5f * (Kr[3 * r + c] - Kr[3 * c + r]);
    float T[9], Kt[9];
    // Kt = V^T Ks V
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) T[3 * r + c] = Ks[3 * r] * V[c] + Ks[3 * r + 1] * V[3 + c] + Ks[3 * r + 2] * V[6 + c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Kt[3 * r + c] = V[r] * T[c] + V[3 + r] * T[3 + c] + V[6 + r] * T[6 + c];
    float Xt[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float den = s[r] + s[c];
            if (fabsf(den) < 1e-6f) den = copysignf(1e-6f, den);
            Xt[3 * r + c] = r == c ? 0.f : Kt[3 * r + c] / den;
        }
    // X = V Xt V^T
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) T[3 * r + c] = V[3 * r] * Xt[c] + V[3 * r + 1] * Xt[3 + c] + V[3 * r + 2] * Xt[6 + c];
    float X[9];
    mul_abt(T, V, X);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Fb[3 * r + c] += 2.f * (R[3 * r] * X[c] + R[3 * r + 1] * X[3 + c] + R[3 * r + 2] * X[6 + c]);
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) m += tb[i] * PFt[i];
    mub = 2.f * m;
    lamb = tr * (J - 1.f) * J;
}

// ------------------------------------------------------------------ seed

// Adjoint of the final state, from caller buffers in scene-major id order
// (bar[0..3] = x, v, C, F; a NULL buffer is zero) to storage order.
struct SeedIn {
    const float* bar[4];
};

__global__ void k_adj_seed(StepArgs a, PState st, SeedIn in, AdjState nxt)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.r.np) return;
    const int i = a.r.p0 + g;
    const size_t cap = a.cap;
    const int gid = a.scenes[scene_of(a, i)].p_begin + st.id[i];
    float* dst[4] = {nxt.x, nxt.v, nxt.C, nxt.F};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int comps = f < 2 ? 3 : 9;
        const float* src = in.bar[f];
        for (int d = 0; d < comps; ++d) dst[f][d * cap + i] = src ? src[comps * (size_t)gid + d] : 0.f;
    }
}

// --------------------------------------------------------------- G2P^-1

__global__ void __launch_bounds__(kAdjThreads) k_g2p_adj(AdjArgs q)
{
    const StepArgs& a = q.a;
    __shared__ __align__(128) float4 vw[2][8 * 64];
    __shared__ float gw[3][kWinNodes];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_item[2];
    const int tid = threadIdx.x;
    const size_t cap = a.cap;
    const int n_act = a.sb.counters[CTR_N_ACT];
    int* work = &a.sb.counters[CTR_WORK_G2P];
    walker_init<kAdjThreads>(a, n_act, vw, bar, s_item, work);
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    for (;;) {
        const int item = s_item[buf];
        if (item >= n_act) break;
        for (int t = tid; t < 3 * kWinNodes; t += kAdjThreads) (&gw[0][0])[t] = 0.f;
        if (!walker_next(a, n_act, vw, bar, s_item, work, buf, phase, item)) return;
        const int start = a.sb.act_start[item], count = a.sb.act_count[item];
        const SceneDev sc = a.scenes[a.sb.act_scene[item]];
        const int n = sc.n, nb = sc.nb, lb = a.sb.act_brick[item] - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float fn = (float)n, dt = a.dt, c4 = 4.f * fn;
        const float4* win = vw[buf];
        for (int k = tid; k < count; k += kAdjThreads) {
            const int s = start + k;
            const int p = a.sb.perm[s];
            int bc[3];
            float f[3], w[9], dw[9];
            particle_weights(a.in.x[p], a.in.x[cap + p], a.in.x[2 * cap + p], n, bc, f, w);
            bspline_d(f[0], dw);
            bspline_d(f[1], dw + 3);
            bspline_d(f[2], dw + 6);
            const int l0 = min(max(bc[0] - ox, 0), 3), l1 = min(max(bc[1] - oy, 0), 3), l2 = min(max(bc[2] - oz, 0), 3);
            // forward recompute of C'
            float B[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) B[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2) {
                        const int wi = l0 + i, wj = l1 + j, wk = l2 + k2;
                        const float4 g = win[(((wi >> 2) << 2) | ((wj >> 2) << 1) | (wk >> 2)) * 64 + (wi & 3) * 16 + (wj & 3) * 4 + (wk & 3)];
                        const float W = w[i] * w[3 + j] * w[6 + k2];
                        const float d[3] = {(float)i - f[0], (float)j - f[1], (float)k2 - f[2]};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            B[c] += W * g.x * d[c];
                            B[3 + c] += W * g.y * d[c];
                            B[6 + c] += W * g.z * d[c];
                        }
                    }
            float Cn[9], F[9], aF[9], aC[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                Cn[i] = c4 * B[i];
                F[i] = a.in.F[i * cap + p];
                aF[i] = q.nxt.F[i * cap + s];
                aC[i] = q.nxt.C[i * cap + s];
            }
            float ax[3], vt[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ax[d] = q.nxt.x[d * cap + s];
                vt[d] = q.nxt.v[d * cap + s] + dt * ax[d];
            }
            // F_bar = (I + dt C')^T F'_bar;  Ct = C'_bar + dt F'_bar F^T
            float Fb[9], Ct[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Fb[3 * r + c] = aF[3 * r + c] + dt * (Cn[r] * aF[c] + Cn[3 + r] * aF[3 + c] + Cn[6 + r] * aF[6 + c]);
                    Ct[3 * r + c] = aC[3 * r + c] + dt * (aF[3 * r] * F[3 * c] + aF[3 * r + 1] * F[3 * c + 1] + aF[3 * r + 2] * F[3 * c + 2]);
                }
            float xb[3] = {ax[0], ax[1], ax[2]};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2) {
                        const int wi = l0 + i, wj = l1 + j, wk = l2 + k2;
                        const float4 g = win[(((wi >> 2) << 2) | ((wj >> 2) << 1) | (wk >> 2)) * 64 + (wi & 3) * 16 + (wj & 3) * 4 + (wk & 3)];
                        const float vI[3] = {g.x, g.y, g.z};
                        const float W = w[i] * w[3 + j] * w[6 + k2];
                        const float gW[3] = {fn * dw[i] * w[3 + j] * w[6 + k2], fn * w[i] * dw[3 + j] * w[6 + k2],
                                             fn * w[i] * w[3 + j] * dw[6 + k2]};
                        const float d[3] = {(float)i - f[0], (float)j - f[1], (float)k2 - f[2]};
                        float Ctd[3], h[3];
#pragma unroll
                        for (int r = 0; r < 3; ++r) Ctd[r] = Ct[3 * r] * d[0] + Ct[3 * r + 1] * d[1] + Ct[3 * r + 2] * d[2];
#pragma unroll
                        for (int c = 0; c < 3; ++c) h[c] = Ct[c] * vI[0] + Ct[3 + c] * vI[1] + Ct[6 + c] * vI[2];
                        const int node = (wi * 6 + wj) * 6 + wk;
#pragma unroll
                        for (int r = 0; r < 3; ++r) atomicAdd(&gw[r][node], W * (vt[r] + c4 * Ctd[r]));
                        const float s1 = vI[0] * (vt[0] + c4 * Ctd[0]) + vI[1] * (vt[1] + c4 * Ctd[1]) + vI[2] * (vt[2] + c4 * Ctd[2]);
#pragma unroll
                        for (int c = 0; c < 3; ++c) xb[c] += gW[c] * s1 - c4 * fn * W * h[c];
                    }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                q.cur.x[d * cap + p] = xb[d];
                q.cur.v[d * cap + p] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                q.cur.F[i * cap + p] = Fb[i];
                q.cur.C[i * cap + p] = 0.f;
            }
        }
        __syncthreads();
        for (int t = tid; t < kWinNodes; t += kAdjThreads) {
            const float g0 = gw[0][t], g1 = gw[1][t], g2 = gw[2][t];
            if (g0 == 0.f && g1 == 0.f && g2 == 0.f) continue;
            const int gi = ox + t / 36, gj = oy + (t / 6) % 6, gk = oz + t % 6;
            if (gi >= n || gj >= n || gk >= n) continue;
            red_add_v4(&a.G[node_index(sc, gi, gj, gk)], g0, g1, g2, 0.f);
        }
        __syncthreads();
        buf ^= 1;
    }
}

// --------------------------------------------------------------- grid^-1
// G holds v_I_bar; V holds the forward (v_I, m_I).  Writes (P_I_bar, m_I_bar)
// into V and clears G.
__global__ void __launch_bounds__(256) k_grid_adj(StepArgs a)
{
    const int tid = threadIdx.x, grp = tid >> 6, nid = tid & 63;
    const int n_nact = a.sb.counters[CTR_N_NACT];
    for (int base = blockIdx.x * 4; base < n_nact; base += gridDim.x * 4) {
        const int item = base + grp;
        if (item >= n_nact) continue;
        const int B = a.sb.nact_brick[item];
        const SceneDev sc = a.scenes[a.sb.nact_scene[item]];
        const int n = sc.n, nb = sc.nb, lb = B - sc.brick_base;
        int bx, by, bz;
        brick_coords(nb, sc.nb_log2, lb, bx, by, bz);
        const int gi = bx * 4 + (nid >> 4);
        const int gj = by * 4 + ((nid >> 2) & 3);
        const int gk = bz * 4 + (nid & 3);
        const int node = B * 64 + nid;
        const float4 vb = a.G[node];
        const float4 vm = a.V[node];
        a.G[node] = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (vm.w > 0.f) {
            float ub[3] = {vb.x, vb.y, vb.z};
            const float v[3] = {vm.x, vm.y, vm.z};
            const int idx[3] = {gi, gj, gk};
            const int lo = a.bound, hi = n - 1 - a.bound;
            if (gj < lo && a.floor_sticky) {
                ub[0] = ub[1] = ub[2] = 0.f;
            } else {
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if ((idx[d] < lo || idx[d] > hi) && v[d] == 0.f) ub[d] = 0.f;  // clamped component
            }
            const float inv = 1.f / vm.w;
            out.x = ub[0] * inv;
            out.y = ub[1] * inv;
            out.z = ub[2] * inv;
            out.w = -(ub[0] * (v[0] - a.dt * a.gravity[0]) + ub[1] * (v[1] - a.dt * a.gravity[1]) +
                      ub[2] * (v[2] - a.dt * a.gravity[2])) * inv;
        }
        a.V[node] = out;
    }
}

// --------------------------------------------------------------- P2G^-1

__global__ void __launch_bounds__(kAdjThreads) k_p2g_adj(AdjArgs q)
{
    const StepArgs& a = q.a;
    __shared__ __align__(128) float4 vw[2][8 * 64];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_item[2];
    const int tid = threadIdx.x;
    const size_t cap = a.cap;
    const int n_act = a.sb.counters[CTR_N_ACT];
    int* work = &a.sb.counters[CTR_WORK_P2G];
    walker_init<kAdjThreads>(a, n_act, vw, bar, s_item, work);
    unsigned phase[2] = {0u, 0u};
    int buf = 0;
    for (;;) {
        const int item = s_item[buf];
        if (item >= n_act) break;
        if (!walker_next(a, n_act, vw, bar, s_item, work, buf, phase, item)) return;
        const int start = a.sb.act_start[item], count = a.sb.act_count[item];
        const int scene = a.sb.act_scene[item];
        const SceneDev sc = a.scenes[scene];
        const int n = sc.n, nb = sc.nb, lb = a.sb.act_brick[item] - sc.brick_base;
        int ox, oy, oz;
        brick_coords(nb, sc.nb_log2, lb, ox, oy, oz);
        ox *= 4; oy *= 4; oz *= 4;
        const float fn = (float)n, dxs = 1.f / fn, m = sc.m_p;
        const float kA = a.dt * sc.V0 * 4.f * fn * fn;
        const float4* win = vw[buf];
        for (int k = tid; k < count; k += kAdjThreads) {
            const int s = start + k;
            const int p = a.sb.perm[s];
            int bc[3];
            float f[3], w[9], dw[9];
            particle_weights(a.in.x[p], a.in.x[cap + p], a.in.x[2 * cap + p], n, bc, f, w);
            bspline_d(f[0], dw);
            bspline_d(f[1], dw + 3);
            bspline_d(f[2], dw + 6);
            const int l0 = min(max(bc[0] - ox, 0), 3), l1 = min(max(bc[1] - oy, 0), 3), l2 = min(max(bc[2] - oz, 0), 3);
            float F[9], C[9], v[3], tau[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                F[i] = a.in.F[i * cap + p];
                C[i] = a.in.C[i * cap + p];
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) v[d] = a.in.v[d * cap + p];
            const float mu = sc.pp_mat ? a.in.mu[p] : sc.mu, lam = sc.pp_mat ? a.in.lam[p] : sc.lam;
            float dummy[9], mub0, lamb0;
            stress_and_vjp(a.model, F, mu, lam, tau, nullptr, dummy, mub0, lamb0);
            float A[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) A[i] = m * C[i] - kA * tau[i];
            float vb[3] = {0.f, 0.f, 0.f}, Ab[9], xb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 9; ++i) Ab[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2) {
                        const int wi = l0 + i, wj = l1 + j, wk = l2 + k2;
                        const float4 g = win[(((wi >> 2) << 2) | ((wj >> 2) << 1) | (wk >> 2)) * 64 + (wi & 3) * 16 + (wj & 3) * 4 + (wk & 3)];
                        const float Pb[3] = {g.x, g.y, g.z};
                        const float mb = g.w;
                        const float W = w[i] * w[3 + j] * w[6 + k2];
                        const float gW[3] = {fn * dw[i] * w[3 + j] * w[6 + k2], fn * w[i] * dw[3 + j] * w[6 + k2],
                                             fn * w[i] * w[3 + j] * dw[6 + k2]};
                        const float d[3] = {((float)i - f[0]) * dxs, ((float)j - f[1]) * dxs, ((float)k2 - f[2]) * dxs};
                        float s2 = m * mb;
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            const float mom = m * v[r] + A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2];
                            s2 += Pb[r] * mom;
                            vb[r] += W * m * Pb[r];
#pragma unroll
                            for (int c = 0; c < 3; ++c) Ab[3 * r + c] += W * Pb[r] * d[c];
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            xb[c] += gW[c] * s2 - W * (A[c] * Pb[0] + A[3 + c] * Pb[1] + A[6 + c] * Pb[2]);
                    }
            float tb[9], Fb[9], mub, lamb;
#pragma unroll
            for (int i = 0; i < 9; ++i) tb[i] = -kA * Ab[i];
            stress_and_vjp(a.model, F, mu, lam, tau, tb, Fb, mub, lamb);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                q.cur.x[d * cap + p] += xb[d];
                q.cur.v[d * cap + p] = vb[d];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                q.cur.C[i * cap + p] = m * Ab[i];
                q.cur.F[i * cap + p] += Fb[i];
            }
            const int gid = sc.p_begin + a.in.id[p];
            q.gmu[gid] += mub;
            q.glam[gid] += lamb;
        }
        __syncthreads();
        buf ^= 1;
    }
}

// ---------------------------------------------------------------- output
// Outputs in scene-major id order: the adjoint of the state at mpm_tape_begin
// (out[0..3] = x, v, C, F; NULL = not wanted) and the gradients with respect to
// the per-particle Young's modulus and Poisson ratio (mu = E / (2(1+nu)),
// lambda = E nu / ((1+nu)(1-2nu))) and Lame parameters.
struct AdjOut {
    float* bar[4];
    float *dE, *dnu, *dmu, *dlam;
};

__global__ void k_adj_out(StepArgs a, PState st0, AdjState adj0, const float* gmu, const float* glam, AdjOut o)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.r.np) return;
    const int i = a.r.p0 + g;
    const size_t cap = a.cap;
    const SceneDev sc = a.scenes[scene_of(a, i)];
    const int gid = sc.p_begin + st0.id[i];
    const float* src[4] = {adj0.x, adj0.v, adj0.C, adj0.F};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!o.bar[f]) continue;
        const int comps = f < 2 ? 3 : 9;
        for (int d = 0; d < comps; ++d) o.bar[f][comps * (size_t)gid + d] = src[f][d * cap + i];
    }
    const float mu = sc.pp_mat ? st0.mu[i] : sc.mu, lam = sc.pp_mat ? st0.lam[i] : sc.lam;
    const float E = mu * (3.f * lam + 2.f * mu) / (lam + mu);
    const float nu = lam / (2.f * (lam + mu));
    const float a1 = 1.f + nu, a2 = 1.f - 2.f * nu;
    const float dmu_dE = 1.f / (2.f * a1), dmu_dnu = -E / (2.f * a1 * a1);
    const float dlam_dE = nu / (a1 * a2), dlam_dnu = E * (1.f + 2.f * nu * nu) / (a1 * a1 * a2 * a2);
    if (o.dE) o.dE[gid] = gmu[gid] * dmu_dE + glam[gid] * dlam_dE;
    if (o.dnu) o.dnu[gid] = gmu[gid] * dmu_dnu + glam[gid] * dlam_dnu;
    if (o.dmu) o.dmu[gid] = gmu[gid];
    if (o.dlam) o.dlam[gid] = glam[gid];
}

}  // namespace mpm

// ================================================================ host

#define MPM_CKA(call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return status_from_cuda(e_);       \
    } while (0)

static int n_blocks(long long n, int t) { return (int)((n + t - 1) / t); }

// staging of host gradient buffers: 24 floats of state adjoint + dE, dnu, dmu, dlam per particle
constexpr int kIoFloats = 28;
static const int kComps[4] = {3, 3, 9, 9};

void mpm_tape_free(mpm_ctx* c)
{
    if (!c || !c->tape) return;
    mpm_tape* t = c->tape;
    for (float* p : t->ckpt) cudaFree(p);
    cudaFree(t->seg);
    cudaFree(t->perms);
    cudaFree(t->adj);
    cudaFree(t->gmat);
    cudaFree(t->io);
    delete t;
    c->tape = nullptr;
}

static int any_rigid(const mpm_ctx* c)
{
    for (const SceneDev& s : c->h_scenes)
        if (s.n_rigid > 0) return 1;
    return 0;
}

extern "C" int mpm_tape_begin(mpm_ctx* c)
{
    if (!c) return MPM_ERR_INVALID_ARGUMENT;
    if (c->cfg.tape_checkpoint_every <= 0 || c->cfg.tape_max_substeps <= 0) return MPM_ERR_STATE;
    if (c->cfg.plasticity != MPM_PLASTIC_NONE || c->cfg.solver != MPM_SOLVER_MLS) return MPM_ERR_STATE;
    int st = upload_scenes(c);
    if (st) return st;
    if ((st = ensure_keys(c))) return st;
    if (!c->tape) {
        mpm_tape* t = new mpm_tape();
        t->K = c->cfg.tape_checkpoint_every;
        t->max_steps = c->cfg.tape_max_substeps;
        t->cap = c->cap;
        c->tape = t;
        const size_t sb = state_bytes(c->cap);
        const int n_ckpt = t->max_steps / t->K + 1;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < n_ckpt && e == cudaSuccess; ++k) {
            float* p = nullptr;
            e = cudaMalloc(&p, sb);
            t->ckpt.push_back(p);
        }
        if (e == cudaSuccess) e = cudaMalloc(&t->seg, sb * (size_t)t->K);
        if (e == cudaSuccess) e = cudaMalloc(&t->perms, sizeof(int) * (size_t)c->cap * t->max_steps);
        if (e == cudaSuccess) e = cudaMalloc(&t->adj, sizeof(float) * 48 * (size_t)c->cap);
        if (e == cudaSuccess) e = cudaMalloc(&t->gmat, sizeof(float) * 2 * (size_t)c->cap);
        if (e == cudaSuccess) e = cudaMalloc(&t->io, sizeof(float) * kIoFloats * (size_t)c->cap);
        if (e != cudaSuccess) {
            mpm_tape_free(c);
            return status_from_cuda(e);
        }
    }
    mpm_tape* t = c->tape;
    // recording runs unfused: start from a clean accumulator
    if (c->g_dirty) MPM_CKA(cudaMemsetAsync(c->G, 0, sizeof(float4) * (size_t)c->total_bricks * 64, c->stream));
    c->g_dirty = false;
    c->g_pending = false;
    MPM_CKA(cudaMemcpyAsync(t->ckpt[0], c->state_mem[c->cur], state_bytes(c->cap), cudaMemcpyDeviceToDevice, c->stream));
    t->dts.clear();
    c->recording = true;
    return MPM_OK;
}

// One recorded substep: the unfused forward, keeping the sort permutation and
// checkpointing every K-th state.
int mpm_tape_record_substep(mpm_ctx* c, float dt)
{
    mpm_tape* t = c->tape;
    if (!t || (int)t->dts.size() >= t->max_steps) return MPM_ERR_STATE;
    const int j = (int)t->dts.size();
    StepArgs a = step_args(c, dt, 0, c->n_scenes, c->st[c->cur], c->st[c->cur ^ 1]);
    a.tau_valid = c->tau_valid;
    int st;
    if ((st = status_from_cuda(launch_sort(a, c->stream)))) return st;
    MPM_CKA(launch_p2g(a, c->stream));
    // the permutation G2P uses (P2G leaves it in cell order inside each pass)
    MPM_CKA(cudaMemcpyAsync(t->perms + (size_t)j * c->cap + a.r.p0, c->sb.perm + a.r.p0, sizeof(int) * a.r.np,
                            cudaMemcpyDeviceToDevice, c->stream));
    MPM_CKA(launch_grid(a, c->stream));
    MPM_CKA(launch_g2p(a, c->stream));
    c->tau_valid = true;
    c->cur ^= 1;
    c->h_time += (double)dt;
    t->dts.push_back(dt);
    if ((int)t->dts.size() % t->K == 0)
        MPM_CKA(cudaMemcpyAsync(t->ckpt[t->dts.size() / t->K], c->state_mem[c->cur], state_bytes(c->cap),
                                cudaMemcpyDeviceToDevice, c->stream));
    return MPM_OK;
}

// Sort bookkeeping of a stored state with a recorded permutation: keys and
// counts from the positions, then the scan (lists, offsets) without a scatter.
static int sort_with_perm(mpm_ctx* c, StepArgs& a, const PState& state, int* perm)
{
    MPM_CKA(reset_histogram(c));
    MPM_CKA(launch_prepare(a, state, c->stream));
    MPM_CKA(launch_sort(a, c->stream, false));
    a.sb.perm = perm;
    return MPM_OK;
}

// Reverse of every recorded substep from the adjoint of the final state
// (seeds, device pointers in id order or NULL) to the adjoint of the state at
// mpm_tape_begin and the material gradients (outputs, device pointers or NULL).
static int backward_device(mpm_ctx* c, const SeedIn& seeds, const AdjOut& outs)
{
    mpm_tape* t = c->tape;
    const int T = (int)t->dts.size();
    const int N = c->total_particles;
    const size_t cap = c->cap;
    int st;
    // the recompute advances the scene clocks; keep them
    std::vector<double> t_save(c->n_scenes);
    std::vector<int> e_save(c->n_scenes);
    if ((st = wait_stream(c))) return st;  // bounded; the copies below then complete at once
    MPM_CKA(cudaMemcpy(t_save.data(), c->d_time, sizeof(double) * c->n_scenes, cudaMemcpyDeviceToHost));
    MPM_CKA(cudaMemcpy(e_save.data(), c->d_epoch, sizeof(int) * c->n_scenes, cudaMemcpyDeviceToHost));

    AdjState adj[2] = {adj_view(t->adj, c->cap), adj_view(t->adj + 24 * cap, c->cap)};
    int nxt = 0;
    MPM_CKA(cudaMemsetAsync(t->gmat, 0, sizeof(float) * 2 * cap, c->stream));
    float* gmu = t->gmat;
    float* glam = t->gmat + cap;
    {
        StepArgs a = step_args(c, 0.f, 0, c->n_scenes, c->st[c->cur], c->st[c->cur]);
        if (N > 0) k_adj_seed<<<n_blocks(N, 256), 256, 0, c->stream>>>(a, c->st[c->cur], seeds, adj[nxt]);
        MPM_CKA(cudaGetLastError());
    }
    const size_t sbytes = state_bytes(c->cap);
    auto seg_state = [&](int k) { return state_view(t->seg + (sbytes / sizeof(float)) * k, c->cap); };
    const int n_seg = T > 0 ? (T - 1) / t->K + 1 : 0;
    for (int sgi = n_seg - 1; sgi >= 0; --sgi) {
        const int j0 = sgi * t->K, j1 = std::min(j0 + t->K, T);
        MPM_CKA(cudaMemcpyAsync(t->seg, t->ckpt[sgi], sbytes, cudaMemcpyDeviceToDevice, c->stream));
        // recompute the segment's states
        for (int j = j0; j < j1 - 1; ++j) {
            StepArgs a = step_args(c, t->dts[j], 0, c->n_scenes, seg_state(j - j0), seg_state(j - j0 + 1));
            a.tau_valid = 0;
            a.cell_order = 0;  // the recorded permutation is already the one G2P used
            if ((st = sort_with_perm(c, a, seg_state(j - j0), t->perms + (size_t)j * cap))) return st;
            MPM_CKA(launch_p2g(a, c->stream));
            MPM_CKA(launch_grid(a, c->stream));
            MPM_CKA(launch_g2p(a, c->stream));
        }
        // reverse the segment's substeps
        for (int j = j1 - 1; j >= j0; --j) {
            StepArgs a = step_args(c, t->dts[j], 0, c->n_scenes, seg_state(j - j0), seg_state(j - j0));
            a.tau_valid = 0;
            a.cell_order = 0;
            if ((st = sort_with_perm(c, a, seg_state(j - j0), t->perms + (size_t)j * cap))) return st;
            MPM_CKA(launch_p2g(a, c->stream));
            MPM_CKA(launch_grid(a, c->stream));
            AdjArgs q{a, adj[nxt], adj[nxt ^ 1], gmu, glam};
            const int ctas = c->num_sms * 2;
            // the walkers fetch work from the G2P and P2G counters: reset them
            MPM_CKA(cudaMemsetAsync(c->sb.counters + CTR_WORK_P2G, 0, sizeof(int) * 3, c->stream));
            k_g2p_adj<<<ctas, kAdjThreads, 0, c->stream>>>(q);
            MPM_CKA(cudaGetLastError());
            k_grid_adj<<<c->num_sms * 8, 256, 0, c->stream>>>(a);
            MPM_CKA(cudaGetLastError());
            k_p2g_adj<<<ctas, kAdjThreads, 0, c->stream>>>(q);
            MPM_CKA(cudaGetLastError());
            nxt ^= 1;
        }
    }
    // outputs (adj[nxt] is the adjoint of the state at mpm_tape_begin)
    const PState st0 = state_view(t->ckpt[0], c->cap);
    StepArgs a = step_args(c, 0.f, 0, c->n_scenes, st0, st0);
    if (N > 0) k_adj_out<<<n_blocks(N, 256), 256, 0, c->stream>>>(a, st0, adj[nxt], gmu, glam, outs);
    MPM_CKA(cudaGetLastError());
    MPM_CKA(cudaMemcpyAsync(c->d_time, t_save.data(), sizeof(double) * c->n_scenes, cudaMemcpyHostToDevice, c->stream));
    MPM_CKA(cudaMemcpyAsync(c->d_epoch, e_save.data(), sizeof(int) * c->n_scenes, cudaMemcpyHostToDevice, c->stream));
    c->keys_valid = false;
    c->tau_valid = false;
    return wait_stream(c);
}

// Shared driver of mpm_backward and mpm_backward_state: stages host buffers
// through the tape's io area (inputs are consumed by the seed kernel before
// any output is written there).
static int backward_common(mpm_ctx* c, const float* const* bar_in, float* const* bar_out, float* dE, float* dnu,
                           float* dmu, float* dlam, int mem)
{
    if (!c || (mem != MPM_MEM_HOST && mem != MPM_MEM_DEVICE)) return MPM_ERR_INVALID_ARGUMENT;
    if (!c->tape || !c->recording) return MPM_ERR_STATE;
    if (any_rigid(c)) return MPM_ERR_STATE;
    mpm_tape* t = c->tape;
    const int N = c->total_particles;
    const size_t cap = c->cap;
    int st = upload_scenes(c);
    if (st) return st;
    SeedIn seeds{};
    AdjOut outs{};
    size_t off[4];
    for (int f = 0, o = 0; f < 4; o += kComps[f], ++f) off[f] = (size_t)o * cap;  // 0, 3, 6, 15 (x cap)
    for (int f = 0; f < 4; ++f) {
        const float* in = bar_in ? bar_in[f] : nullptr;
        if (in && mem == MPM_MEM_HOST) {
            float* d = t->io + off[f];
            MPM_CKA(cudaMemcpyAsync(d, in, sizeof(float) * kComps[f] * N, cudaMemcpyHostToDevice, c->stream));
            in = d;
        }
        seeds.bar[f] = in;
        float* out = bar_out ? bar_out[f] : nullptr;
        outs.bar[f] = (out && mem == MPM_MEM_HOST) ? t->io + off[f] : out;
    }
    float* host_scalar[4] = {dE, dnu, dmu, dlam};
    float** dev_scalar[4] = {&outs.dE, &outs.dnu, &outs.dmu, &outs.dlam};
    for (int k = 0; k < 4; ++k)
        *dev_scalar[k] = (host_scalar[k] && mem == MPM_MEM_HOST) ? t->io + (24 + k) * cap : host_scalar[k];
    if ((st = backward_device(c, seeds, outs))) return st;
    if (mem == MPM_MEM_HOST) {
        for (int f = 0; f < 4; ++f)
            if (bar_out && bar_out[f])
                MPM_CKA(cudaMemcpy(bar_out[f], outs.bar[f], sizeof(float) * kComps[f] * N, cudaMemcpyDeviceToHost));
        for (int k = 0; k < 4; ++k)
            if (host_scalar[k]) MPM_CKA(cudaMemcpy(host_scalar[k], *dev_scalar[k], sizeof(float) * N, cudaMemcpyDeviceToHost));
    }
    return MPM_OK;
}

extern "C" int mpm_backward(mpm_ctx* c, const float* dLdx, const float* dLdv, float* dLdE, float* dLdnu,
                            float* dLdv0, int mem)
{
    const float* in[4] = {dLdx, dLdv, nullptr, nullptr};
    float* out[4] = {nullptr, dLdv0, nullptr, nullptr};
    return backward_common(c, in, out, dLdE, dLdnu, nullptr, nullptr, mem);
}

extern "C" int mpm_backward_state(mpm_ctx* c, const float* const* bar_in, float* const* bar_out, float* dL_dmu,
                                  float* dL_dlam, int mem)
{
    return backward_common(c, bar_in, bar_out, nullptr, nullptr, dL_dmu, dL_dlam, mem);
}
