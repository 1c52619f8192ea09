// Device-side data layout and math of the MLS-MPM substep (arXiv 2502.18437,
// Sec. III-B, Algorithm 1) for sm_103a.
//
// Layout in HBM
//  - particles: structure of arrays, component-major: x[3][cap], v[3][cap],
//    C[9][cap], F[9][cap], tau[6][cap], mu[cap], lam[cap], id[cap].  Two copies ping-pong:
//    each substep reads one through the sort permutation and G2P writes the
//    other in sorted order, so particles stay sorted by brick in storage.
//  - grid: each scene owns a dense block of (n/4)^3 bricks of 4^3 nodes;
//    brick (bx,by,bz) of scene s is global brick brick_base[s] +
//    (bx*nb + by)*nb + bz and node (lx,ly,lz) of a brick is at
//    brick*64 + lx*16 + ly*4 + lz.  P2G accumulates float4 (m, mv) per node;
//    the grid update writes float4 (v, m) to a second array.  Only bricks
//    touched by particles are ever processed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm.h"

namespace mpm {

constexpr int kMaxRigids = MPM_MAX_RIGIDS;
constexpr int kMaxPts = MPM_MAX_SEGMENT_POINTS;
constexpr int kWin = 6;                    // P2G/G2P node window per brick: 4 + 2
constexpr int kWinNodes = kWin * kWin * kWin;

struct SceneDev {
    int n;           // nodes per dimension
    int nb;          // bricks per dimension
    int brick_base;  // first global brick of the scene
    int p_begin;     // first particle (storage index)
    int p_count;     // number of particles
    int pp_mat;      // 1: per-particle mu/lam arrays
    int n_rigid;     // rigid slots in use
    int tile_base;   // first scan tile of the scene (tiles never straddle scenes)
    float m_p, V0;   // particle mass and initial volume
    float mu, lam;   // uniform Lame parameters (pp_mat == 0)
    int nb_log2;     // log2(nb) when nb is a power of two, else -1
};

// Coordinates (bx, by, bz) of the scene-local brick lb = (bx nb + by) nb + bz:
// shifts for power-of-two grids, divisions otherwise.
__device__ __forceinline__ void brick_coords(int nb, int nb_log2, int lb, int& bx, int& by, int& bz)
{
    if (nb_log2 >= 0) {
        bx = lb >> (2 * nb_log2);
        by = (lb >> nb_log2) & (nb - 1);
        bz = lb & (nb - 1);
    } else {
        bx = lb / (nb * nb);
        by = (lb / nb) % nb;
        bz = lb % nb;
    }
}

constexpr int kMaxTris = MPM_MAX_MESH_TRIANGLES;
constexpr int kMaxSpine = MPM_MAX_SPINE_POINTS;

// Shape data shared by the device copy and the staged pose: segment points or
// mesh vertices (body frame) and the mesh's triangles and spine polyline.
struct RigidShape {
    float pts[kMaxPts * 3];
    unsigned char tris[kMaxTris * 3];  // vertex indices (< kMaxPts)
    unsigned char spine[kMaxSpine];
};

struct RigidDev {
    int type, n_pts, n_tris, n_spine;
    float c0[3], q0[4], vel[3], omega[3];
    float mu_k, c_d, margin, radius;
    float half[3];
    float thickness, spine_radius;
    double t_set;    // scene time at which (c0, q0) was the pose
    RigidShape shape;
};

// Pose of a rigid at the current scene time, staged in shared memory.
struct RigidCur {
    int type, n_pts, n_tris, n_spine;
    float c[3], R[9], vel[3], omega[3];
    float mu_k, c_d, margin, radius;
    float half[3];
    float thickness, spine_radius;
    RigidShape shape;
};

// Pose of a solid rigid (sphere, box) at the end of the substep, for the
// particle push-out at the end of G2P.
struct SolidPose {
    int type;
    float c[3], R[9];
    float radius;
    float half[3];
};

struct PState {
    float* x;
    float* v;
    float* C;
    float* F;
    float* tau;  // Kirchhoff stress of F (xx xy xz yy yz zz), written by the unfused G2P
    float* mu;
    float* lam;
    int* id;
};

// Counters shared by the kernels of one substep.
enum {
    CTR_N_ACT = 0,     // active particle bricks
    CTR_N_NACT = 1,    // active node bricks
    CTR_DONE_G2P = 2,  // CTAs of the G2P launch that have finished (the last one advances the clocks)
    CTR_WORK_P2G = 3,  // dynamic work counters of the persistent kernels
    CTR_WORK_GRID = 4,
    CTR_WORK_G2P = 5,
    CTR_COUNT = 8
};

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ float3 f3(float a, float b, float c) { return make_float3(a, b, c); }

// Base cell of a coordinate: floor(x*n - 0.5) with one rounding, clamped to
// [0, n-3] so that the 3-node stencil stays on the grid (NaN maps to 0).
// Returns 1 when clamping was needed (particle outside the grid).
__device__ __forceinline__ int base_cell(float x, int n, int& b)
{
    float s = floorf(__fmaf_rn(x, (float)n, -0.5f));
    if (!(s >= 0.0f)) { b = 0; return 1; }
    if (s > (float)(n - 3)) { b = n - 3; return 1; }
    b = (int)s;
    return 0;
}

__device__ __forceinline__ void bspline(float f, float w[3])
{
    // quadratic B-spline at distances f, f-1, f-2 (f in [0.5, 1.5))
    float a = 1.5f - f, b = f - 1.0f, c = f - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}

// Derivatives of the three quadratic B-spline weights with respect to f
// (the basis gradient of the standard MPM's Eq. 2 and Eq. 5 is n times these).
__device__ __forceinline__ void bspline_d(float f, float dw[3])
{
    dw[0] = f - 1.5f;
    dw[1] = -2.0f * (f - 1.0f);
    dw[2] = f - 0.5f;
}

__device__ __forceinline__ float det3(const float F[9])
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// ------------------------------------------------------------- 3x3 SVD
//
// (The adjoint's decomposition; the forward constitutive update uses the
// closed-form sym_eigen3 below.)
// Rotation-variant SVD F = U diag(s) V^T (det U = det V = +1, s sorted by
// decreasing magnitude, s[2] < 0 when det F < 0) in FP32, after McAdams et al.
// 2011 ("Computing the SVD of 3x3 matrices with minimal branching"): cyclic
// Jacobi eigen-analysis of the symmetric F^T F for V (here with the textbook
// Givens tangent rather than approximate quaternion rotations, 4 sweeps), sorting of the columns of B = F V, and a Givens QR of B
// for U and s, which recovers small singular values accurately from B rather
// than from the squared eigenvalues.

__device__ __forceinline__ float approx_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// One Jacobi rotation of the symmetric (p,q) block, annihilating a_pq.  With
// d = a_qq - a_pp and b = 2 a_pq the textbook tangent of the smaller angle,
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)) with theta = d/b, equals
// sign(d) b / (|d| + sqrt(d^2 + b^2)); the rotation is (c, s) = (1, t)/sqrt(1+t^2),
// exactly orthogonal up to rounding whatever the accuracy of t.
__device__ __forceinline__ void jacobi_rot(float& app, float& aqq, float& apq, float& arp, float& arq,
                                           float& v0p, float& v0q, float& v1p, float& v1q, float& v2p,
                                           float& v2q)
{
    // converged: an off-diagonal below half a unit roundoff of the larger diagonal
    // entry (2^-25) is smaller than the rounding error of that entry itself, so the
    // rotation would not change the result in single precision (this also keeps
    // b^2 clear of underflow)
    if (!(fabsf(apq) > 2.98e-8f * fmaxf(fabsf(app), fabsf(aqq)))) return;
    const float d = aqq - app, b = 2.0f * apq;
    // |d| + sqrt(d^2 + b^2) >= |b| > 0; the max keeps that true where b^2 underflows
    // (only for a degenerate F, whose entries would be below ~1e-9)
    const float den = fmaxf(fabsf(d) + approx_sqrt(__fmaf_rn(d, d, b * b)), fabsf(b));
    const float t = __fdividef(d >= 0.0f ? b : -b, den);
    const float c = rsqrtf(__fmaf_rn(t, t, 1.0f));
    const float s = t * c;
    app = __fmaf_rn(-t, apq, app);
    aqq = __fmaf_rn(t, apq, aqq);
    apq = 0.0f;
    float rp = c * arp - s * arq, rq = s * arp + c * arq;
    arp = rp;
    arq = rq;
    float x, y;
    x = v0p; y = v0q; v0p = c * x - s * y; v0q = s * x + c * y;
    x = v1p; y = v1q; v1p = c * x - s * y; v1q = s * x + c * y;
    x = v2p; y = v2q; v2p = c * x - s * y; v2q = s * x + c * y;
}

__device__ __forceinline__ void swap_neg_cols(float M[9], int i, int j)
{
    // swap columns i and j and negate the new column j (keeps the determinant)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float t = M[3 * r + i];
        M[3 * r + i] = M[3 * r + j];
        M[3 * r + j] = -t;
    }
}

__device__ __forceinline__ void givens_rows(float B[9], float U[9], int i, int k)
{
    // rotate rows i,k of B to zero B[k][i]; U accumulates the transpose
    float a = B[3 * i + i], b = B[3 * k + i];
    float r2 = __fmaf_rn(a, a, b * b);
    float c = 1.0f, s = 0.0f;
    if (r2 > 1e-37f) {
        float inv = rsqrtf(r2);
        c = a * inv;
        s = b * inv;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float bi = B[3 * i + j], bk = B[3 * k + j];
        B[3 * i + j] = c * bi + s * bk;
        B[3 * k + j] = -s * bi + c * bk;
        float ui = U[3 * j + i], uk = U[3 * j + k];
        U[3 * j + i] = c * ui + s * uk;
        U[3 * j + k] = -s * ui + c * uk;
    }
}

__device__ __forceinline__ void svd3(const float F[9], float U[9], float s[3], float V[9])
{
    float a00 = F[0] * F[0] + F[3] * F[3] + F[6] * F[6];
    float a01 = F[0] * F[1] + F[3] * F[4] + F[6] * F[7];
    float a02 = F[0] * F[2] + F[3] * F[5] + F[6] * F[8];
    float a11 = F[1] * F[1] + F[4] * F[4] + F[7] * F[7];
    float a12 = F[1] * F[2] + F[4] * F[5] + F[7] * F[8];
    float a22 = F[2] * F[2] + F[5] * F[5] + F[8] * F[8];
#pragma unroll
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
#pragma unroll
    for (int sweep = 0; sweep < 4; ++sweep) {
        jacobi_rot(a00, a11, a01, a02, a12, V[0], V[1], V[3], V[4], V[6], V[7]);
        jacobi_rot(a00, a22, a02, a01, a12, V[0], V[2], V[3], V[5], V[6], V[8]);
        jacobi_rot(a11, a22, a12, a01, a02, V[1], V[2], V[4], V[5], V[7], V[8]);
    }
    float B[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            B[3 * r + c] = F[3 * r] * V[c] + F[3 * r + 1] * V[3 + c] + F[3 * r + 2] * V[6 + c];
    // sort by decreasing eigenvalue of F^T F
    if (a00 < a11) { swap_neg_cols(B, 0, 1); swap_neg_cols(V, 0, 1); float t = a00; a00 = a11; a11 = t; }
    if (a00 < a22) { swap_neg_cols(B, 0, 2); swap_neg_cols(V, 0, 2); float t = a00; a00 = a22; a22 = t; }
    if (a11 < a22) { swap_neg_cols(B, 1, 2); swap_neg_cols(V, 1, 2); float t = a11; a11 = a22; a22 = t; }
#pragma unroll
    for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
    givens_rows(B, U, 0, 1);
    givens_rows(B, U, 0, 2);
    givens_rows(B, U, 1, 2);
    s[0] = B[0];
    s[1] = B[4];
    s[2] = B[8];
}

// Eigen-decomposition A = U diag(l) U^T of a symmetric 3x3 matrix in closed
// form, after Eberly's robust 3x3 symmetric eigensolver: the characteristic
// cubic of the deviator B = A - q I (q = tr A / 3) in its trigonometric form
// (Smith 1961, the cosine solved here from the trisection cubic) gives the
// eigenvalue farthest from the other two (the largest when det B >= 0, else
// the smallest), whose eigenvector is the longest cross
// product of two rows of A - l I; the 2x2 block of B in an orthonormal basis of
// that vector's complement is then diagonalised by one exact Jacobi rotation.
// Working on B keeps the rounding at the scale of the deviator's entries, and
// the first eigenvalue is taken from its eigenvector (Rayleigh quotient).  The
// columns of U are orthonormal to rounding (det U may be -1).  A deviator at
// the rounding level of A (or a non-finite A) gives U = I and the diagonal.
__device__ __forceinline__ void sym_eigen3(float a00, float a01, float a02, float a11, float a12, float a22,
                                           float U[9], float l[3])
{
    const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * (a01 * a01 + a02 * a02 + a12 * a12);
#pragma unroll
    for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
    l[0] = a00;
    l[1] = a11;
    l[2] = a22;
    if (!(p2 > 1e-13f * q * q)) return;
    const float p = sqrtf(p2 * (1.0f / 6.0f));
    const float ip = 1.0f / p;
    const float c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    // det(B / p) / 2 = cos(3 phi); the eigenvalues are q + 2 p cos(phi + 2 pi k / 3).
    // The one farthest from the others is q + 2 p c with c the largest root of the
    // trisection cubic 4 c^3 - 3 c = |r| (in [cos(pi/6), 1]), signed like r (the
    // cubic is odd): two Newton steps from the chord reach FP32 rounding.
    const float det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
    const float r = fminf(fmaxf(0.5f * det, -1.0f), 1.0f);
    const float t = fabsf(r);
    float c = 0.8660254f + 0.1339746f * t;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const float c2 = c * c;
        c -= __fdividef(__fmaf_rn(4.0f, c2, -3.0f) * c - t, __fmaf_rn(12.0f, c2, -3.0f));
    }
    const float d1 = copysignf(2.0f * p * c, r);  // l1 - q
    const float m00 = b00 - d1, m11 = b11 - d1, m22 = b22 - d1;
    // the longest cross product of two rows of A - l1 I
    float e0 = a01 * a12 - a02 * m11, e1 = a02 * a01 - m00 * a12, e2 = m00 * m11 - a01 * a01;
    float nn = e0 * e0 + e1 * e1 + e2 * e2;
    {
        const float x = a01 * m22 - a02 * a12, y = a02 * a02 - m00 * m22, z = m00 * a12 - a01 * a02;
        const float n2 = x * x + y * y + z * z;
        if (n2 > nn) { e0 = x; e1 = y; e2 = z; nn = n2; }
    }
    {
        const float x = m11 * m22 - a12 * a12, y = a12 * a02 - a01 * m22, z = a01 * a12 - m11 * a02;
        const float n2 = x * x + y * y + z * z;
        if (n2 > nn) { e0 = x; e1 = y; e2 = z; nn = n2; }
    }
    if (!(nn > 0.0f)) return;
    const float in = rsqrtf(nn);
    const float v0 = e0 * in, v1 = e1 * in, v2 = e2 * in;
    // orthonormal u, w with (v, u, w) a right-handed basis
    float u0, u1, u2;
    if (fabsf(v0) > fabsf(v1)) {
        const float k = rsqrtf(v0 * v0 + v2 * v2);
        u0 = -v2 * k; u1 = 0.0f; u2 = v0 * k;
    } else {
        const float k = rsqrtf(v1 * v1 + v2 * v2);
        u0 = 0.0f; u1 = v2 * k; u2 = -v1 * k;
    }
    const float w0 = v1 * u2 - v2 * u1, w1 = v2 * u0 - v0 * u2, w2 = v0 * u1 - v1 * u0;
    // B v, B u, B w
    const float bv0 = b00 * v0 + a01 * v1 + a02 * v2, bv1 = a01 * v0 + b11 * v1 + a12 * v2,
                bv2 = a02 * v0 + a12 * v1 + b22 * v2;
    const float bu0 = b00 * u0 + a01 * u1 + a02 * u2, bu1 = a01 * u0 + b11 * u1 + a12 * u2,
                bu2 = a02 * u0 + a12 * u1 + b22 * u2;
    const float bw0 = b00 * w0 + a01 * w1 + a02 * w2, bw1 = a01 * w0 + b11 * w1 + a12 * w2,
                bw2 = a02 * w0 + a12 * w1 + b22 * w2;
    const float muu = u0 * bu0 + u1 * bu1 + u2 * bu2, muw = w0 * bu0 + w1 * bu1 + w2 * bu2,
                mww = w0 * bw0 + w1 * bw1 + w2 * bw2;
    l[0] = q + (v0 * bv0 + v1 * bv1 + v2 * bv2);
    // the 2x2 block [[muu, muw], [muw, mww]]: one rotation (textbook tangent of
    // the smaller angle, as in jacobi_rot)
    float cr = 1.0f, sr = 0.0f, tm = 0.0f;
    if (fabsf(muw) > 2.98e-8f * fmaxf(fabsf(muu + q), fabsf(mww + q))) {
        const float d = mww - muu, b = 2.0f * muw;
        const float den = fmaxf(fabsf(d) + approx_sqrt(__fmaf_rn(d, d, b * b)), fabsf(b));
        const float t = __fdividef(d >= 0.0f ? b : -b, den);
        cr = rsqrtf(__fmaf_rn(t, t, 1.0f));
        sr = t * cr;
        tm = t * muw;
    }
    l[1] = q + (muu - tm);
    l[2] = q + (mww + tm);
    U[0] = v0; U[3] = v1; U[6] = v2;
    U[1] = cr * u0 - sr * w0; U[4] = cr * u1 - sr * w1; U[7] = cr * u2 - sr * w2;
    U[2] = sr * u0 + cr * w0; U[5] = sr * u1 + cr * w1; U[8] = sr * u2 + cr * w2;
}

// Left stretch of F for the constitutive update: the eigen-decomposition
// F F^T = U diag(l) U^T (closed form, sym_eigen3) and the signed singular
// values of the rotation-variant SVD F = U diag(s) V^T.  The two larger are
// sqrt(l); the smallest is det F / (their product), signed like det F and
// accurate where sqrt of a tiny eigenvalue of F F^T is not.  V is never formed:
// the stress needs U and s only, and the plastic return map is
// F' = U diag(s'/s) U^T F; neither depends on the signs of U's columns.
__device__ __forceinline__ void left_stretch(const float F[9], float U[9], float s[3])
{
    float l[3];
    sym_eigen3(F[0] * F[0] + F[1] * F[1] + F[2] * F[2], F[0] * F[3] + F[1] * F[4] + F[2] * F[5],
               F[0] * F[6] + F[1] * F[7] + F[2] * F[8], F[3] * F[3] + F[4] * F[4] + F[5] * F[5],
               F[3] * F[6] + F[4] * F[7] + F[5] * F[8], F[6] * F[6] + F[7] * F[7] + F[8] * F[8], U, l);
    const float a00 = l[0], a11 = l[1], a22 = l[2];
    const float J = det3(F);
    const float r0 = approx_sqrt(a00), r1 = approx_sqrt(a11), r2 = approx_sqrt(a22);
    // smallest eigenvalue: its singular value from the determinant
    const int m = (a00 <= a11 && a00 <= a22) ? 0 : (a11 <= a22 ? 1 : 2);
    const float pa = m == 0 ? r1 * r2 : (m == 1 ? r0 * r2 : r0 * r1);
    const float sm = pa > 1e-30f ? __fdividef(J, pa) : 0.0f;
    s[0] = m == 0 ? sm : r0;
    s[1] = m == 1 ? sm : r1;
    s[2] = m == 2 ? sm : r2;
}

// R = U V^T
__device__ __forceinline__ void mul_abt(const float A[9], const float B[9], float out[9])
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            out[3 * r + c] = A[3 * r] * B[3 * c] + A[3 * r + 1] * B[3 * c + 1] + A[3 * r + 2] * B[3 * c + 2];
}

// ------------------------------------------------------------ stresses
//
// Constitutive update of one particle, the last step of the G2P loop of
// Algorithm 1: optional plastic projection of F, then the Kirchhoff stress
// tau = J sigma of the (projected) F, stored symmetric as (xx xy xz yy yz zz).
// The paper's Eq. 6 is the Cauchy form; with V = J V0 the P2G force term
// V sigma equals V0 tau.
//  - fixed-corotated: tau = 2 mu (F - R) F^T + lambda (J - 1) J I with R the
//    rotation of the polar decomposition.  With F = U S V^T (rotation-variant
//    SVD) and R = U V^T this is U diag(2 mu (s - 1) s) U^T + lambda (J-1) J I.
//  - Neo-Hookean: tau = mu (F F^T - I) + lambda ln(J) I (J <= 0: flagged).
//  - von Mises on the Hencky strain (plasticity is the paper's future work;
//    the law is the library's definition): eps = ln s, dev = eps - tr(eps)/3,
//    gamma = |dev| - yield / (2 mu); when gamma > 0, eps -= gamma dev/|dev| and
//    F = U diag(exp eps) V^T.
// Returns error bits.
__device__ __forceinline__ unsigned constitutive(int model, int plastic, float yield, float mu, float lam,
                                                 float F[9], float t6[6])
{
    unsigned e = 0u;
    if (model == MPM_FIXED_COROTATED || plastic) {
        float U[9], s[3];
        left_stretch(F, U, s);
        if (plastic) {
            if (!(s[0] > 0.0f && s[1] > 0.0f && s[2] > 0.0f)) {
                e |= MPM_EBIT_INVERTED;
            } else {
                const float e0 = __logf(s[0]), e1 = __logf(s[1]), e2 = __logf(s[2]);
                const float tr = (e0 + e1 + e2) * (1.0f / 3.0f);
                const float d0 = e0 - tr, d1 = e1 - tr, d2 = e2 - tr;
                const float nrm = approx_sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                const float gamma = nrm - __fdividef(yield, 2.0f * mu);
                if (gamma > 0.0f && nrm > 0.0f) {
                    const float k = __fdividef(gamma, nrm);
                    const float n0 = __expf(e0 - k * d0), n1 = __expf(e1 - k * d1), n2 = __expf(e2 - k * d2);
                    // F' = U diag(s'/s) U^T F = U diag(s') V^T
                    const float q0 = __fdividef(n0, s[0]), q1 = __fdividef(n1, s[1]), q2 = __fdividef(n2, s[2]);
                    float M[9];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = r; c < 3; ++c) {
                            M[3 * r + c] = U[3 * r] * q0 * U[3 * c] + U[3 * r + 1] * q1 * U[3 * c + 1] +
                                           U[3 * r + 2] * q2 * U[3 * c + 2];
                            M[3 * c + r] = M[3 * r + c];
                        }
                    float Fp[9];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            Fp[3 * r + c] = M[3 * r] * F[c] + M[3 * r + 1] * F[3 + c] + M[3 * r + 2] * F[6 + c];
#pragma unroll
                    for (int i = 0; i < 9; ++i) F[i] = Fp[i];
                    s[0] = n0;
                    s[1] = n1;
                    s[2] = n2;
                }
            }
        }
        if (model == MPM_FIXED_COROTATED) {
            const float J = s[0] * s[1] * s[2];
            const float l = lam * (J - 1.0f) * J;
            const float g0 = 2.0f * mu * (s[0] - 1.0f) * s[0];
            const float g1 = 2.0f * mu * (s[1] - 1.0f) * s[1];
            const float g2 = 2.0f * mu * (s[2] - 1.0f) * s[2];
            // U diag(g) U^T + l I
            t6[0] = g0 * U[0] * U[0] + g1 * U[1] * U[1] + g2 * U[2] * U[2] + l;
            t6[1] = g0 * U[0] * U[3] + g1 * U[1] * U[4] + g2 * U[2] * U[5];
            t6[2] = g0 * U[0] * U[6] + g1 * U[1] * U[7] + g2 * U[2] * U[8];
            t6[3] = g0 * U[3] * U[3] + g1 * U[4] * U[4] + g2 * U[5] * U[5] + l;
            t6[4] = g0 * U[3] * U[6] + g1 * U[4] * U[7] + g2 * U[5] * U[8];
            t6[5] = g0 * U[6] * U[6] + g1 * U[7] * U[7] + g2 * U[8] * U[8] + l;
            return e;
        }
    }
    const float J = det3(F);
    float lnJ = 0.0f;
    if (J > 0.0f) lnJ = __logf(J);
    else e |= MPM_EBIT_INVERTED;
    const float d = __fmaf_rn(lam, lnJ, -mu);
    t6[0] = mu * (F[0] * F[0] + F[1] * F[1] + F[2] * F[2]) + d;
    t6[1] = mu * (F[0] * F[3] + F[1] * F[4] + F[2] * F[5]);
    t6[2] = mu * (F[0] * F[6] + F[1] * F[7] + F[2] * F[8]);
    t6[3] = mu * (F[3] * F[3] + F[4] * F[4] + F[5] * F[5]) + d;
    t6[4] = mu * (F[3] * F[6] + F[4] * F[7] + F[5] * F[8]);
    t6[5] = mu * (F[6] * F[6] + F[7] * F[7] + F[8] * F[8]) + d;
    return e;
}

// Co-rotational material constraint of PB-MPM (Sec. III-C) for one particle,
// in place of the stress in P2G: F* = (I + dt C) F, R its polar rotation,
// F* <- beta R + (1 - beta) F* / det(F*) (as printed), C <- (F* F^-1 - I) / dt.
// R = U diag(s)^-1 U^T F* from the left stretch of F* (F* = U diag(s) V^T with
// U, V rotations, so R = U V^T).
__device__ __forceinline__ void pb_constraint(const float F[9], float dt, float beta, float C[9])
{
    float Fh[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Fh[3 * r + c] = F[3 * r + c] + dt * (C[3 * r] * F[c] + C[3 * r + 1] * F[3 + c] + C[3 * r + 2] * F[6 + c]);
    float U[9], s[3];
    left_stretch(Fh, U, s);
    const float i0 = 1.0f / s[0], i1 = 1.0f / s[1], i2 = 1.0f / s[2];
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            M[3 * r + c] = U[3 * r] * i0 * U[3 * c] + U[3 * r + 1] * i1 * U[3 * c + 1] + U[3 * r + 2] * i2 * U[3 * c + 2];
            M[3 * c + r] = M[3 * r + c];
        }
    const float k = (1.0f - beta) / det3(Fh);
    float Fs[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Fs[3 * r + c] = beta * (M[3 * r] * Fh[c] + M[3 * r + 1] * Fh[3 + c] + M[3 * r + 2] * Fh[6 + c]) +
                            k * Fh[3 * r + c];
    // F^-1 = adj(F) / det(F)
    const float id = 1.0f / det3(F);
    const float Fi[9] = {(F[4] * F[8] - F[5] * F[7]) * id, (F[2] * F[7] - F[1] * F[8]) * id,
                         (F[1] * F[5] - F[2] * F[4]) * id, (F[5] * F[6] - F[3] * F[8]) * id,
                         (F[0] * F[8] - F[2] * F[6]) * id, (F[2] * F[3] - F[0] * F[5]) * id,
                         (F[3] * F[7] - F[4] * F[6]) * id, (F[1] * F[6] - F[0] * F[7]) * id,
                         (F[0] * F[4] - F[1] * F[3]) * id};
    const float idt = 1.0f / dt;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = ((Fs[3 * r] * Fi[c] + Fs[3 * r + 1] * Fi[3 + c] + Fs[3 * r + 2] * Fi[6 + c]) -
                            (r == c ? 1.0f : 0.0f)) * idt;
}

// Rotation matrix of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_mat(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

}  // namespace mpm
