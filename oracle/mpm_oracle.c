/*
 * FP64 CPU oracle of one MLS-MPM substep (CRESSim-MPM, arXiv 2502.18437).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle_mpm.so and is
 * loaded by the test-suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark.  The CUDA library never links, loads or calls it, and the two share
 * no code, header, table or helper.
 *
 * The oracle is the paper's Algorithm 1 (Sec. III-B, "APIC-style MLS-MPM
 * simulation step") run serially in double precision on a dense n^3 grid:
 *   particle loop : P2G mass (Eq. 1, first part) and fused momentum/force (Eq. 8)
 *   node loop     : velocity update with gravity (Eq. 3), contact (Sec. IV, Eq. 11,
 *                   Eq. 12) and domain boundaries
 *   particle loop : affine transfer (Eq. 9), advection (Eq. 4), deformation
 *                   gradient (Eq. 10), constitutive update
 *   reset grid; rigid poses advance; particles left inside solid rigids are
 *   pushed out to the surface (Sec. IV-A).
 * Passages the paper leaves open are resolved by the reading written at the
 * function that needs it.  No blocking, fusion or reordering is done beyond the
 * order of Algorithm 1.
 *
 * Conventions: domain [0,1)^3, dx = 1/n, node I at I*dx, row-major 3x3 matrices,
 * node (i,j,k) stored at (i*n + j)*n + k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_PTS 64
#define ORC_MAX_TRIS 64
#define ORC_MAX_SPINE 16
#define ORC_TWO_PI 6.283185307179586476925286766559

enum { ORC_ERR_OUT_OF_DOMAIN = 1, ORC_ERR_NONFINITE = 2, ORC_ERR_INVERTED = 4 };
enum { ORC_FIXED_COROTATED = 0, ORC_NEO_HOOKEAN = 1 };
enum { ORC_SPHERE = 0, ORC_BOX = 1, ORC_QUAD_SLICER = 2, ORC_SEGMENTS = 3, ORC_ARC = 4, ORC_MESH_SLICER = 5 };
enum { ORC_REGION_NONE = 0, ORC_REGION_REGULAR = 1, ORC_REGION_ONED = 2, ORC_REGION_STICKY = 3 };

typedef struct {
    int n;              /* grid nodes per dimension, dx = 1/n */
    int bound;          /* boundary width in nodes */
    int floor_sticky;   /* y-low boundary: 1 sticky, 0 slip */
    int model;          /* ORC_FIXED_COROTATED or ORC_NEO_HOOKEAN */
    int plasticity;     /* 0 none, 1 von Mises on the Hencky strain */
    int pad_;
    double yield_stress;
    double gravity[3];
    double m_p;         /* particle mass */
    double V0;          /* particle initial volume */
} orc_config;

typedef struct {
    int type;
    int n_pts;
    double c[3];        /* centre, world frame */
    double R[9];        /* body -> world rotation, row-major */
    double vel[3];      /* linear velocity of the centre */
    double omega[3];    /* angular velocity, world frame */
    double mu_k, c_d, margin;
    double radius;      /* sphere radius; segment (capsule) radius */
    double half[3];     /* box half extents; slicer: half[0] along the edge, half[1] spine->edge */
    double thickness;   /* slicer thickness */
    double spine_radius;/* slicer spine circle radius */
    double pts[ORC_MAX_PTS * 3]; /* segment chain points / mesh vertices, body frame */
    double impulse[6];  /* accumulated momentum given to the rigid: linear, angular about c */
    /* arc: half[0] circle radius, half[1] start angle, half[2] sweep (radians, in
       the body x-y plane, centred on the body origin); radius = wire radius */
    int n_tris, n_spine;             /* mesh slicer: triangles, spine polyline points */
    int tris[ORC_MAX_TRIS * 3];      /* vertex indices into pts */
    int spine[ORC_MAX_SPINE];        /* vertex indices of the spine polyline */
} orc_rigid;

/* ---------------------------------------------------------------- helpers */

static double det3(const double A[9])
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void matmul3(const double A[9], const double B[9], double out[9])
{
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(out, t, sizeof t);
}

/* A * B^T */
static void matmul3_bt(const double A[9], const double B[9], double out[9])
{
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * j + k];
            t[3 * i + j] = s;
        }
    memcpy(out, t, sizeof t);
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    out[0] = t0; out[1] = t1; out[2] = t2;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------- shape function */

/* Quadratic B-spline basis N(r) (Sec. III-A: finite support, 3 nodes per
 * dimension), written as its textbook piecewise definition. */
double orc_bspline_N(double r)
{
    double a = fabs(r);
    if (a < 0.5) return 0.75 - a * a;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

/* Weights of the 3 nodes base, base+1, base+2 for the fractional offset
 * f = x/dx - base, base = floor(x/dx - 0.5), so f lies in [0.5, 1.5). */
void orc_bspline_weights(double f, double w[3])
{
    for (int i = 0; i < 3; ++i) w[i] = orc_bspline_N(f - (double)i);
}

/* ----------------------------------------------------------------- SVD */

/* Singular value decomposition A = U diag(S) V^T by one-sided (Hestenes)
 * Jacobi rotations, run to convergence in double precision.  Rotation-variant
 * convention: det U = det V = +1 and the smallest singular value carries the
 * sign of det A (so an inverted A has S[2] < 0).  S is sorted by decreasing
 * magnitude of the unsigned values. */
void orc_svd3(const double A[9], double U[9], double S[3], double V[9])
{
    double W[9];
    memcpy(W, A, sizeof W);
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    static const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int k = 0; k < 3; ++k) {
            int p = pairs[k][0], q = pairs[k][1];
            double alpha = 0, beta = 0, gamma = 0;
            for (int i = 0; i < 3; ++i) {
                alpha += W[3 * i + p] * W[3 * i + p];
                beta += W[3 * i + q] * W[3 * i + q];
                gamma += W[3 * i + p] * W[3 * i + q];
            }
            if (gamma == 0.0 || fabs(gamma) <= 1e-17 * sqrt(alpha * beta)) continue;
            double zeta = (beta - alpha) / (2.0 * gamma);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
            for (int i = 0; i < 3; ++i) {
                double wp = W[3 * i + p], wq = W[3 * i + q];
                W[3 * i + p] = c * wp - s * wq;
                W[3 * i + q] = s * wp + c * wq;
                double vp = V[3 * i + p], vq = V[3 * i + q];
                V[3 * i + p] = c * vp - s * vq;
                V[3 * i + q] = s * vp + c * vq;
            }
            rotated = 1;
        }
        if (!rotated) break;
    }
    double sig[3];
    for (int j = 0; j < 3; ++j) sig[j] = sqrt(W[j] * W[j] + W[3 + j] * W[3 + j] + W[6 + j] * W[6 + j]);
    /* sort columns by decreasing singular value */
    int order[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (sig[order[b]] > sig[order[a]]) { int t = order[a]; order[a] = order[b]; order[b] = t; }
    double Ws[9], Vs[9];
    for (int j = 0; j < 3; ++j) {
        S[j] = sig[order[j]];
        for (int i = 0; i < 3; ++i) {
            Ws[3 * i + j] = W[3 * i + order[j]];
            Vs[3 * i + j] = V[3 * i + order[j]];
        }
    }
    memcpy(V, Vs, sizeof Vs);
    /* U columns = W columns / sigma; complete the basis where sigma vanishes */
    double scale = S[0] > 0 ? S[0] : 1.0;
    for (int j = 0; j < 3; ++j) {
        if (S[j] > 1e-300 && S[j] > 1e-14 * scale) {
            for (int i = 0; i < 3; ++i) U[3 * i + j] = Ws[3 * i + j] / S[j];
        } else {
            double col[3];
            if (j == 0) { col[0] = 1; col[1] = 0; col[2] = 0; }
            else if (j == 1) {
                /* any unit vector orthogonal to column 0 */
                double u0[3] = {U[0], U[3], U[6]};
                double e[3] = {fabs(u0[0]) < 0.9 ? 1.0 : 0.0, fabs(u0[0]) < 0.9 ? 0.0 : 1.0, 0.0};
                cross3(u0, e, col);
                double l = sqrt(dot3(col, col));
                for (int i = 0; i < 3; ++i) col[i] /= l;
            } else {
                double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]};
                cross3(u0, u1, col);
            }
            for (int i = 0; i < 3; ++i) U[3 * i + j] = col[i];
        }
    }
    if (det3(U) < 0) { for (int i = 0; i < 3; ++i) U[3 * i + 2] = -U[3 * i + 2]; S[2] = -S[2]; }
    if (det3(V) < 0) { for (int i = 0; i < 3; ++i) V[3 * i + 2] = -V[3 * i + 2]; S[2] = -S[2]; }
}

/* Rotation factor of the polar decomposition A = R S (the PolarDecomp of
 * Sec. III-C), R = U V^T with the rotation-variant SVD above, so det R = +1. */
void orc_polar_R(const double A[9], double R[9])
{
    double U[9], S[3], V[9];
    orc_svd3(A, U, S, V);
    matmul3_bt(U, V, R);
}

/* --------------------------------------------------------------- stress */

/* Kirchhoff stress tau = J sigma.
 * Neo-Hookean: Eq. 6 multiplied by J, tau = mu (F F^T - I) + lambda ln(J) I; the
 *   paper notes that implementations may use the Kirchhoff stress directly.
 *   J <= 0 has no logarithm: reported as ORC_ERR_INVERTED, tau left at zero.
 * Fixed-corotated (the elastic law of the workloads; not printed in the paper):
 *   tau = 2 mu (F - R) F^T + lambda (J - 1) J I, R from the polar decomposition.
 * Returns error bits. */
int orc_kirchhoff(int model, const double F[9], double mu, double lam, double tau[9])
{
    double J = det3(F);
    if (model == ORC_NEO_HOOKEAN) {
        if (!(J > 0.0)) { memset(tau, 0, 9 * sizeof(double)); return ORC_ERR_INVERTED; }
        double FFt[9];
        matmul3_bt(F, F, FFt);
        double lnJ = log(J);
        for (int i = 0; i < 9; ++i) tau[i] = mu * (FFt[i] - ((i % 4 == 0) ? 1.0 : 0.0));
        for (int i = 0; i < 3; ++i) tau[4 * i] += lam * lnJ;
        return 0;
    }
    double R[9], FmR[9], P[9];
    orc_polar_R(F, R);
    for (int i = 0; i < 9; ++i) FmR[i] = F[i] - R[i];
    matmul3_bt(FmR, F, P);
    for (int i = 0; i < 9; ++i) tau[i] = 2.0 * mu * P[i];
    for (int i = 0; i < 3; ++i) tau[4 * i] += lam * (J - 1.0) * J;
    return 0;
}

/* Kirchhoff stress of N particles (tau: N x 9); returns the OR of error bits. */
int orc_kirchhoff_all(int model, int N, const double* F, const double* mu, const double* lam, double* tau)
{
    int err = 0;
    for (int p = 0; p < N; ++p) err |= orc_kirchhoff(model, F + 9 * p, mu[p], lam[p], tau + 9 * p);
    return err;
}

/* Lame parameters from Young's modulus and Poisson ratio (textbook). */
void orc_lame(double E, double nu, double* mu, double* lam)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* ----------------------------------------------------------- plasticity */

/* Von Mises return mapping on the Hencky (logarithmic) strain.  The paper
 * lists elastoplastic materials as future work (Sec. VI) and prints no law,
 * so this is a definitional choice: F = U diag(s) V^T, eps = ln s,
 * eps_hat = eps - tr(eps)/3, gamma = |eps_hat| - yield/(2 mu); when gamma > 0,
 * eps -= gamma eps_hat/|eps_hat| and F = U diag(exp eps) V^T.  A singular
 * value <= 0 has no logarithm: reported as ORC_ERR_INVERTED, F unchanged.
 * Returns error bits. */
int orc_von_mises(double F[9], double mu, double yield)
{
    double U[9], s[3], V[9];
    orc_svd3(F, U, s, V);
    if (!(s[2] > 0.0)) return ORC_ERR_INVERTED;
    double eps[3] = {log(s[0]), log(s[1]), log(s[2])};
    double tr = (eps[0] + eps[1] + eps[2]) / 3.0;
    double eh[3] = {eps[0] - tr, eps[1] - tr, eps[2] - tr};
    double norm = sqrt(dot3(eh, eh));
    double gamma = norm - yield / (2.0 * mu);
    if (gamma <= 0.0 || norm == 0.0) return 0;
    for (int i = 0; i < 3; ++i) eps[i] -= gamma * eh[i] / norm;
    double US[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) US[3 * i + j] = U[3 * i + j] * exp(eps[j]);
    matmul3_bt(US, V, F);
    return 0;
}

/* ------------------------------------------------------ rigid geometry */

void orc_rigid_set_quat(orc_rigid* r, const double q_in[4])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    double* R = r->R;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Kinematic pose advance over one substep: the rigid moves with its set
 * velocities (the host solver sets them between steps, Sec. V-C).
 * Rotation by Rodrigues' formula for the angle |omega| dt. */
void orc_rigid_advance(orc_rigid* r, double dt)
{
    for (int i = 0; i < 3; ++i) r->c[i] += dt * r->vel[i];
    double w = sqrt(dot3(r->omega, r->omega));
    if (w == 0.0) return;
    double th = w * dt, k[3] = {r->omega[0] / w, r->omega[1] / w, r->omega[2] / w};
    double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0}, K2[9], Rot[9];
    matmul3(K, K, K2);
    for (int i = 0; i < 9; ++i) Rot[i] = ((i % 4 == 0) ? 1.0 : 0.0) + sin(th) * K[i] + (1.0 - cos(th)) * K2[i];
    matmul3(Rot, r->R, r->R);
}

static void to_world(const orc_rigid* r, const double a[3], double out[3])
{
    for (int i = 0; i < 3; ++i) out[i] = r->R[3 * i] * a[0] + r->R[3 * i + 1] * a[1] + r->R[3 * i + 2] * a[2];
}

/* Nearest point q of segment [a, b] to p (endpoint projections keep the
 * segment); returns |p - q|. */
static double closest_on_segment(const double p[3], const double a[3], const double b[3], double q[3])
{
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double L2 = dot3(ab, ab);
    double u = L2 > 0 ? dot3(ap, ab) / L2 : 0.0;
    if (u < 0) u = 0;
    if (u > 1) u = 1;
    for (int i = 0; i < 3; ++i) q[i] = a[i] + u * ab[i];
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    return sqrt(dot3(d, d));
}

/* Nearest point q of triangle (a, b, c) to p: the orthogonal projection when it
 * falls inside (barycentric coordinates from the 2x2 normal equations of the
 * plane's least-squares problem; *interior = 1), else the nearest of the three
 * edges' nearest points (*interior = 0).  Returns |p - q|. */
static double closest_on_triangle(const double p[3], const double a[3], const double b[3], const double c[3],
                                  double q[3], int* interior)
{
    double e0[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e1[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double d00 = dot3(e0, e0), d01 = dot3(e0, e1), d11 = dot3(e1, e1), d20 = dot3(ap, e0), d21 = dot3(ap, e1);
    double den = d00 * d11 - d01 * d01;
    *interior = 0;
    if (den > 0) {
        double s = (d11 * d20 - d01 * d21) / den, t = (d00 * d21 - d01 * d20) / den;
        if (s >= 0 && t >= 0 && s + t <= 1) {
            for (int i = 0; i < 3; ++i) q[i] = a[i] + s * e0[i] + t * e1[i];
            double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
            *interior = 1;
            return sqrt(dot3(d, d));
        }
    }
    double qa[3], qb[3], qc[3];
    double da = closest_on_segment(p, a, b, qa), db = closest_on_segment(p, b, c, qb), dc = closest_on_segment(p, c, a, qc);
    double best = da;
    memcpy(q, qa, sizeof qa);
    if (db < best) { best = db; memcpy(q, qb, sizeof qb); }
    if (dc < best) { best = dc; memcpy(q, qc, sizeof qc); }
    return best;
}

/* Nearest point of the arc (circle of radius Ra about the body origin in the
 * body x-y plane, angles th0 .. th0 + sweep) to the body point p, and the unit
 * tangent there (direction of increasing angle).  A point on the circle's
 * axis has every angle at the same distance and takes the start angle. */
static double closest_on_arc(const double p[3], double Ra, double th0, double sweep, double q[3], double t[3])
{
    double th;
    if (p[0] == 0.0 && p[1] == 0.0) {
        th = th0;
    } else {
        double phi = atan2(p[1], p[0]);
        double rel = fmod(phi - th0, ORC_TWO_PI);
        if (rel < 0) rel += ORC_TWO_PI;
        if (rel <= sweep) {
            th = th0 + rel;
        } else {
            /* outside the sweep: the nearer endpoint */
            double qe0[3] = {Ra * cos(th0), Ra * sin(th0), 0.0};
            double qe1[3] = {Ra * cos(th0 + sweep), Ra * sin(th0 + sweep), 0.0};
            double d0[3] = {p[0] - qe0[0], p[1] - qe0[1], p[2]}, d1[3] = {p[0] - qe1[0], p[1] - qe1[1], p[2]};
            th = dot3(d1, d1) < dot3(d0, d0) ? th0 + sweep : th0;
        }
    }
    q[0] = Ra * cos(th); q[1] = Ra * sin(th); q[2] = 0.0;
    t[0] = -sin(th); t[1] = cos(th); t[2] = 0.0;
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    return sqrt(dot3(d, d));
}

/* Region test and contact frame of one rigid at world point xw.
 * Returns the region code; n (unit normal, world) and t (unit tangent, world,
 * ONED only) are filled when the code is not NONE; *dist receives the distance
 * used by the region test.  Readings:
 *  - solid shapes (sphere, box): node in contact when sdf < margin; normal is
 *    the outward SDF gradient;
 *  - slicer (Sec. IV-B): the blade is the planar quad |s|<=a, |t|<=b, eta=0 of
 *    thickness h in body frame (s along body x = edge direction, t along body y
 *    pointing from the spine to the edge, eta along body z).  The spine is the
 *    segment t=-b with a circular distance field; a node closer than
 *    spine_radius + margin to it gets sticky contact.  Otherwise a node with
 *    |sdf| = distance to the quad below h/2 + margin gets regular contact with
 *    normal sign(eta) n_q on the faces (eta = 0 counts as +) and the direction
 *    from the nearest quad point off the faces;
 *  - connected segments (Sec. IV-C): 1D geometry; nearest segment wins (ties
 *    to the lower index); node in contact when the distance is below
 *    radius + margin; n from the projected point to the node, t along the
 *    segment.  A node on the centre line has no normal: n is left zero.
 *  - arc (Sec. IV-C, the suture needle): 1D geometry like the segments, with
 *    the arc's tangent at the nearest point as t;
 *  - triangle-mesh slicer (Sec. IV-B): a blade given as an open triangle mesh
 *    of thickness h and a spine polyline.  A node closer than spine_radius +
 *    margin to the spine gets sticky contact; otherwise a node closer than
 *    h/2 + margin to the nearest triangle (lowest index on ties) gets regular
 *    contact with normal sign((x - q) . n_T) n_T where its nearest point q lies
 *    inside the triangle (0 counts as +), and (x - q)/|x - q| off it. */
int orc_geometry(const orc_rigid* r, const double xw[3], double n[3], double t[3], double* dist)
{
    double d[3] = {xw[0] - r->c[0], xw[1] - r->c[1], xw[2] - r->c[2]}, p[3];
    for (int i = 0; i < 3; ++i) p[i] = r->R[i] * d[0] + r->R[3 + i] * d[1] + r->R[6 + i] * d[2];
    double nl[3] = {0, 0, 0}, tl[3] = {0, 0, 0};
    int code = ORC_REGION_NONE;
    if (r->type == ORC_SPHERE) {
        double l = sqrt(dot3(p, p));
        *dist = l - r->radius;
        if (*dist < r->margin) {
            code = ORC_REGION_REGULAR;
            if (l > 0) { nl[0] = p[0] / l; nl[1] = p[1] / l; nl[2] = p[2] / l; }
            else nl[1] = 1.0;
        }
    } else if (r->type == ORC_BOX) {
        double q[3], qo[3];
        for (int i = 0; i < 3; ++i) { q[i] = fabs(p[i]) - r->half[i]; qo[i] = q[i] > 0 ? q[i] : 0.0; }
        double outside = sqrt(dot3(qo, qo));
        double mx = q[0] > q[1] ? (q[0] > q[2] ? q[0] : q[2]) : (q[1] > q[2] ? q[1] : q[2]);
        *dist = outside + (mx < 0 ? mx : 0.0);
        if (*dist < r->margin) {
            code = ORC_REGION_REGULAR;
            if (outside > 0) {
                for (int i = 0; i < 3; ++i) nl[i] = (p[i] >= 0 ? 1.0 : -1.0) * qo[i] / outside;
            } else {
                int ax = 0;
                for (int i = 1; i < 3; ++i) if (q[i] > q[ax]) ax = i;
                nl[ax] = p[ax] >= 0 ? 1.0 : -1.0;
            }
        }
    } else if (r->type == ORC_QUAD_SLICER) {
        double a = r->half[0], b = r->half[1];
        double es = fabs(p[0]) - a; if (es < 0) es = 0;
        double et = p[1] + b;
        double dsp = sqrt(es * es + et * et + p[2] * p[2]);
        if (dsp < r->spine_radius + r->margin) {
            *dist = dsp;
            code = ORC_REGION_STICKY;
        } else {
            double qs = p[0] < -a ? -a : (p[0] > a ? a : p[0]);
            double qt = p[1] < -b ? -b : (p[1] > b ? b : p[1]);
            double dv[3] = {p[0] - qs, p[1] - qt, p[2]};
            double l = sqrt(dot3(dv, dv));
            *dist = l;
            if (l < 0.5 * r->thickness + r->margin) {
                code = ORC_REGION_REGULAR;
                if (fabs(p[0]) <= a && fabs(p[1]) <= b) nl[2] = p[2] >= 0 ? 1.0 : -1.0;
                else { nl[0] = dv[0] / l; nl[1] = dv[1] / l; nl[2] = dv[2] / l; }
            }
        }
    } else if (r->type == ORC_ARC) {
        double q[3], tt[3];
        double l = closest_on_arc(p, r->half[0], r->half[1], r->half[2], q, tt);
        *dist = l;
        if (l < r->radius + r->margin) {
            code = ORC_REGION_ONED;
            if (l > 0) for (int i = 0; i < 3; ++i) nl[i] = (p[i] - q[i]) / l;
            memcpy(tl, tt, sizeof tl);
        }
    } else if (r->type == ORC_MESH_SLICER) {
        double dsp = INFINITY;
        for (int k = 0; k + 1 < r->n_spine; ++k) {
            double q[3];
            double l = closest_on_segment(p, r->pts + 3 * r->spine[k], r->pts + 3 * r->spine[k + 1], q);
            if (l < dsp) dsp = l;
        }
        if (dsp < r->spine_radius + r->margin) {
            *dist = dsp;
            code = ORC_REGION_STICKY;
        } else {
            double best = INFINITY, bq[3] = {0, 0, 0};
            int bt = -1, binside = 0;
            for (int k = 0; k < r->n_tris; ++k) {
                double q[3];
                int inside;
                const int* tv = r->tris + 3 * k;
                double l = closest_on_triangle(p, r->pts + 3 * tv[0], r->pts + 3 * tv[1], r->pts + 3 * tv[2], q, &inside);
                if (l < best) { best = l; memcpy(bq, q, sizeof bq); bt = k; binside = inside; }
            }
            *dist = best;
            if (bt >= 0 && best < 0.5 * r->thickness + r->margin) {
                code = ORC_REGION_REGULAR;
                if (binside) {
                    const int* tv = r->tris + 3 * bt;
                    const double* a = r->pts + 3 * tv[0];
                    const double* b = r->pts + 3 * tv[1];
                    const double* c = r->pts + 3 * tv[2];
                    double e0[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e1[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
                    double nt[3];
                    cross3(e0, e1, nt);
                    double ln = sqrt(dot3(nt, nt));
                    double dp[3] = {p[0] - bq[0], p[1] - bq[1], p[2] - bq[2]};
                    double sg = dot3(dp, nt) >= 0 ? 1.0 : -1.0;
                    for (int i = 0; i < 3; ++i) nl[i] = sg * nt[i] / ln;
                } else if (best > 0) {
                    for (int i = 0; i < 3; ++i) nl[i] = (p[i] - bq[i]) / best;
                }
            }
        }
    } else if (r->type == ORC_SEGMENTS) {
        double best = INFINITY, bq[3] = {0, 0, 0}, bt[3] = {0, 0, 0};
        for (int s = 0; s + 1 < r->n_pts; ++s) {
            const double* a = r->pts + 3 * s;
            const double* b = r->pts + 3 * (s + 1);
            double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
            double L2 = dot3(ab, ab);
            double u = L2 > 0 ? dot3(ap, ab) / L2 : 0.0;
            if (u < 0) u = 0;
            if (u > 1) u = 1;
            double q[3] = {a[0] + u * ab[0], a[1] + u * ab[1], a[2] + u * ab[2]};
            double dv[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
            double l = sqrt(dot3(dv, dv));
            if (l < best) {
                best = l;
                memcpy(bq, q, sizeof bq);
                double L = sqrt(L2);
                for (int i = 0; i < 3; ++i) bt[i] = L > 0 ? ab[i] / L : 0.0;
            }
        }
        *dist = best;
        if (best < r->radius + r->margin) {
            code = ORC_REGION_ONED;
            if (best > 0) for (int i = 0; i < 3; ++i) nl[i] = (p[i] - bq[i]) / best;
            memcpy(tl, bt, sizeof tl);
        }
    }
    to_world(r, nl, n);
    to_world(r, tl, t);
    return code;
}

/* Contact correction of one node's velocity v (in place) against rigid r,
 * Sec. IV-A to IV-C.  v_rel = v - v_r(x), v_r = vel + omega x (x - c).
 *  - STICKY (slicer spine): v'_rel = 0.
 *  - REGULAR: v_n = v_rel . n; separating when v_n >= 0 (unchanged); else
 *    v_tg = v_rel - v_n n and Eq. 11 read with the Coulomb sign,
 *    v'_rel = c_d max(1 - mu_k |v_n| / |v_tg|, 0) v_tg  (zero when |v_tg| = 0).
 *  - ONED (Eq. 12): same with v_tg replaced by v_tg1 = (v_rel . t) t; a node
 *    on the centre line (no normal) is treated as approaching with v_n = 0.
 * The momentum change of the node, m (v' - v), is given with opposite sign to
 * the rigid (two-way coupling, Sec. IV-A and V-C); linear and angular (about
 * the rigid centre) parts are accumulated in r->impulse. */
void orc_contact_node(orc_rigid* r, const double xI[3], double mI, double v[3])
{
    double n[3], t[3], dist;
    int code = orc_geometry(r, xI, n, t, &dist);
    if (code == ORC_REGION_NONE) return;
    double rx[3] = {xI[0] - r->c[0], xI[1] - r->c[1], xI[2] - r->c[2]}, wr[3];
    cross3(r->omega, rx, wr);
    double vr[3] = {r->vel[0] + wr[0], r->vel[1] + wr[1], r->vel[2] + wr[2]};
    double vrel[3] = {v[0] - vr[0], v[1] - vr[1], v[2] - vr[2]};
    double vnew[3];
    if (code == ORC_REGION_STICKY) {
        vnew[0] = vnew[1] = vnew[2] = 0.0;
    } else {
        double vn = dot3(vrel, n);
        int has_normal = dot3(n, n) > 0.0;
        if (has_normal && vn >= 0.0) return; /* separating */
        if (!has_normal) vn = 0.0;
        double vt[3];
        if (code == ORC_REGION_REGULAR) {
            for (int i = 0; i < 3; ++i) vt[i] = vrel[i] - vn * n[i];
        } else {
            double a = dot3(vrel, t);
            for (int i = 0; i < 3; ++i) vt[i] = a * t[i];
        }
        double lt = sqrt(dot3(vt, vt));
        double scale = 0.0;
        if (lt > 0.0) {
            scale = 1.0 - r->mu_k * fabs(vn) / lt;
            if (scale < 0.0) scale = 0.0;
            scale *= r->c_d;
        }
        for (int i = 0; i < 3; ++i) vnew[i] = scale * vt[i];
    }
    double dp[3];
    for (int i = 0; i < 3; ++i) {
        dp[i] = mI * (vnew[i] - vrel[i]);
        v[i] = vr[i] + vnew[i];
        r->impulse[i] -= dp[i];
    }
    double ang[3];
    cross3(rx, dp, ang);
    for (int i = 0; i < 3; ++i) r->impulse[3 + i] -= ang[i];
}

/* Particle push-out (Sec. IV-A): after the grid-level contact, particles that
 * still ended the substep inside a rigid are pushed out of it, after the
 * particle collision step of Stomakhin et al. 2013.  Reading: this applies to
 * the solid shapes (sphere, box), evaluated at the rigid's pose at the end of
 * the substep; a particle with sdf(x) < 0 is moved to the nearest surface
 * point, x <- x - sdf(x) n(x) with n the outward SDF gradient, in rigid-id
 * order; its velocity, C and F stay as the transfers made them, and no
 * momentum is booked to the rigid.  Blades and line segments push nothing
 * out: the tissue is meant to close around them (Sec. IV-B, IV-C).
 * Returns 1 when x moved. */
int orc_push_out(const orc_rigid* r, double x[3])
{
    if (r->type != ORC_SPHERE && r->type != ORC_BOX) return 0;
    double n[3], t[3], dist;
    int code = orc_geometry(r, x, n, t, &dist);
    if (code == ORC_REGION_NONE || !(dist < 0.0)) return 0;
    for (int i = 0; i < 3; ++i) x[i] -= dist * n[i];
    return 1;
}

/* ------------------------------------------------------------ the step */

static int base_and_frac(const orc_config* cfg, const double xp[3], int b[3], double f[3])
{
    int err = 0;
    for (int d = 0; d < 3; ++d) {
        double s = xp[d] * cfg->n;
        b[d] = (int)floor(s - 0.5);
        if (!(b[d] >= 0 && b[d] + 2 <= cfg->n - 1)) err = ORC_ERR_OUT_OF_DOMAIN;
        f[d] = s - b[d];
    }
    return err;
}

/* P2G (Algorithm 1, first particle loop).
 * Mass: m_I += N_I(x_p) m_p (Eq. 1).  Momentum (Eq. 8 together with the APIC
 * particle momentum m_p v_p that the printed equation omits, as in the cited
 * MLS-MPM formulation): (mv)_I += N_I (m_p v_p + (m_p C_p - dt V0 M^-1 tau_p)(x_I - x_p))
 * with M^-1 = 4/dx^2 (Eq. 7) and V sigma = V0 tau (V = J V0, Eq. 5).
 * gm: n^3 masses, gmv: n^3 x 3 momenta, both accumulated into (caller zeroes).
 * Particles whose stencil leaves the grid are skipped and flagged. */
int orc_p2g(const orc_config* cfg, int N, const double* x, const double* v, const double* C,
            const double* F, const double* mu, const double* lam, double dt, double* gm, double* gmv)
{
    int err = 0, n = cfg->n;
    double dx = 1.0 / n, Minv = 4.0 / (dx * dx);
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) orc_bspline_weights(f[d], w[d]);
        double tau[9], A[9];
        err |= orc_kirchhoff(cfg->model, F + 9 * p, mu[p], lam[p], tau);
        for (int i = 0; i < 9; ++i) A[i] = cfg->m_p * C[9 * p + i] - dt * cfg->V0 * Minv * tau[i];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double dpos[3] = {(b[0] + i) * dx - x[3 * p], (b[1] + j) * dx - x[3 * p + 1],
                                      (b[2] + k) * dx - x[3 * p + 2]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    gm[I] += W * cfg->m_p;
                    for (int r = 0; r < 3; ++r)
                        gmv[3 * I + r] += W * (cfg->m_p * v[3 * p + r] + A[3 * r] * dpos[0] +
                                               A[3 * r + 1] * dpos[1] + A[3 * r + 2] * dpos[2]);
                }
    }
    return err;
}

/* Grid update (Algorithm 1, node loop).  For m_I > 0: v_I = (mv)_I / m_I + dt g
 * (Eq. 3 with f_ext = sum N m g), then each rigid in index order (Sec. IV), then
 * the domain boundary: nodes within `bound` of a face are walls; the y-low
 * wall is sticky (v = 0) when floor_sticky, every other wall removes the
 * velocity component pointing into it.  Nodes with m_I = 0 get v_I = 0.
 * gmv holds momentum on entry and velocity on exit. */
int orc_grid_update(const orc_config* cfg, const double* gm, double* gmv, int n_rigid,
                    orc_rigid* rigids, double dt)
{
    int n = cfg->n;
    double dx = 1.0 / n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                int64_t I = ((int64_t)i * n + j) * n + k;
                double* v = gmv + 3 * I;
                if (!(gm[I] > 0.0)) { v[0] = v[1] = v[2] = 0.0; continue; }
                for (int d = 0; d < 3; ++d) v[d] = v[d] / gm[I] + dt * cfg->gravity[d];
                double xI[3] = {i * dx, j * dx, k * dx};
                for (int r = 0; r < n_rigid; ++r) orc_contact_node(&rigids[r], xI, gm[I], v);
                int idx[3] = {i, j, k};
                for (int d = 0; d < 3; ++d) {
                    if (idx[d] < cfg->bound) {
                        if (d == 1 && cfg->floor_sticky) { v[0] = v[1] = v[2] = 0.0; }
                        else if (v[d] < 0.0) v[d] = 0.0;
                    }
                    if (idx[d] > n - 1 - cfg->bound && v[d] > 0.0) v[d] = 0.0;
                }
            }
    return 0;
}

/* G2P (Algorithm 1, second particle loop): v_p = sum N_I v_I (Eq. 4),
 * B_p = sum N_I v_I (x_I - x_p)^T and C_p = B_p D^-1 with D = dx^2/4 I (Eq. 9),
 * x_p += dt v_p (Eq. 4), F_p = (I + dt C_p) F_p (Eq. 10), then the plastic
 * projection when enabled.  gv: n^3 x 3 node velocities. */
int orc_g2p(const orc_config* cfg, int N, double* x, double* v, double* C, double* F,
            const double* mu, double dt, const double* gv)
{
    int err = 0, n = cfg->n;
    double dx = 1.0 / n, Dinv = 4.0 / (dx * dx);
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) orc_bspline_weights(f[d], w[d]);
        double vp[3] = {0, 0, 0}, B[9] = {0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double dpos[3] = {(b[0] + i) * dx - x[3 * p], (b[1] + j) * dx - x[3 * p + 1],
                                      (b[2] + k) * dx - x[3 * p + 2]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    for (int r = 0; r < 3; ++r) {
                        vp[r] += W * gv[3 * I + r];
                        for (int c = 0; c < 3; ++c) B[3 * r + c] += W * gv[3 * I + r] * dpos[c];
                    }
                }
        double Cn[9], G[9];
        for (int i = 0; i < 9; ++i) Cn[i] = Dinv * B[i];
        for (int i = 0; i < 9; ++i) G[i] = ((i % 4 == 0) ? 1.0 : 0.0) + dt * Cn[i];
        matmul3(G, F + 9 * p, F + 9 * p);
        if (cfg->plasticity) err |= orc_von_mises(F + 9 * p, mu[p], cfg->yield_stress);
        for (int r = 0; r < 3; ++r) {
            v[3 * p + r] = vp[r];
            x[3 * p + r] += dt * vp[r];
        }
        memcpy(C + 9 * p, Cn, sizeof Cn);
        for (int i = 0; i < 3; ++i) if (!isfinite(x[3 * p + i]) || !isfinite(v[3 * p + i])) err |= ORC_ERR_NONFINITE;
        for (int i = 0; i < 9; ++i) if (!isfinite(F[9 * p + i])) err |= ORC_ERR_NONFINITE;
    }
    return err;
}

/* One full substep (Algorithm 1): P2G, grid update, G2P, reset grid, the
 * kinematic advance of the rigids, and the push-out of particles left inside
 * solid rigids.  grid: caller-provided scratch of n^3 x 4
 * doubles (mass + 3 momentum/velocity); on return it holds the node masses in
 * [0, n^3) and node velocities after the grid update in [n^3, 4 n^3) (the
 * reset of Algorithm 1 happens at the start of the next call). */
int orc_substep(const orc_config* cfg, int N, double* x, double* v, double* C, double* F,
                const double* mu, const double* lam, int n_rigid, orc_rigid* rigids, double dt,
                double* grid)
{
    int64_t nn = (int64_t)cfg->n * cfg->n * cfg->n;
    memset(grid, 0, (size_t)nn * 4 * sizeof(double));
    double* gm = grid;
    double* gmv = grid + nn;
    int err = orc_p2g(cfg, N, x, v, C, F, mu, lam, dt, gm, gmv);
    if (err & ORC_ERR_OUT_OF_DOMAIN) return err;
    err |= orc_grid_update(cfg, gm, gmv, n_rigid, rigids, dt);
    err |= orc_g2p(cfg, N, x, v, C, F, mu, dt, gmv);
    for (int r = 0; r < n_rigid; ++r) orc_rigid_advance(&rigids[r], dt);
    for (int p = 0; p < N; ++p)
        for (int r = 0; r < n_rigid; ++r) orc_push_out(&rigids[r], x + 3 * p);
    return err;
}

/* n_steps substeps; allocates its own grid.  Stops at the first error. */
int orc_run(const orc_config* cfg, int N, double* x, double* v, double* C, double* F,
            const double* mu, const double* lam, int n_rigid, orc_rigid* rigids, double dt,
            int n_steps)
{
    int64_t nn = (int64_t)cfg->n * cfg->n * cfg->n;
    double* grid = (double*)malloc((size_t)nn * 4 * sizeof(double));
    if (!grid) return -1;
    int err = 0;
    for (int s = 0; s < n_steps && !err; ++s)
        err = orc_substep(cfg, N, x, v, C, F, mu, lam, n_rigid, rigids, dt, grid);
    free(grid);
    return err;
}

/* ------------------------------------------------------- standard MPM */

/* Derivative dN/dr of the quadratic B-spline basis (textbook piecewise). */
double orc_bspline_dN(double r)
{
    double a = fabs(r);
    if (a < 0.5) return -2.0 * r;
    if (a < 1.5) return (r > 0 ? -1.0 : 1.0) * (1.5 - a);
    return 0.0;
}

/* Weights and their derivatives (w.r.t. the particle coordinate in cell
 * units) of the 3 nodes base, base+1, base+2. */
static void bspline_w_dw(double f, double w[3], double dw[3])
{
    for (int i = 0; i < 3; ++i) {
        w[i] = orc_bspline_N(f - (double)i);
        dw[i] = orc_bspline_dN(f - (double)i);
    }
}

/* P2G of the standard MPM (Sec. III-A), PIC-style: m_I += phi m (Eq. 1),
 * (m v)_I += phi m v (Eq. 1) plus the internal-force impulse dt f_I^int with
 * f_I^int = -sum V sigma grad phi (Eq. 2), V sigma = V0 tau (V = J V0), so the
 * momentum entering Eq. 3 is (m v)_I - dt V0 tau grad phi_I(x_p).  grad phi is
 * the spatial gradient, (1/dx) times the derivative in cell units.  External
 * force: gravity, added in the grid update as v_I += dt g (Eq. 3 with
 * f_ext = m_I g).  gm, gmv accumulated into (caller zeroes). */
int orc_p2g_standard(const orc_config* cfg, int N, const double* x, const double* v, const double* F,
                     const double* mu, const double* lam, double dt, double* gm, double* gmv)
{
    int err = 0, n = cfg->n;
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3], dw[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) bspline_w_dw(f[d], w[d], dw[d]);
        double tau[9];
        err |= orc_kirchhoff(cfg->model, F + 9 * p, mu[p], lam[p], tau);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double gW[3] = {n * dw[0][i] * w[1][j] * w[2][k], n * w[0][i] * dw[1][j] * w[2][k],
                                    n * w[0][i] * w[1][j] * dw[2][k]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    gm[I] += W * cfg->m_p;
                    for (int r = 0; r < 3; ++r)
                        gmv[3 * I + r] += W * cfg->m_p * v[3 * p + r] -
                                          dt * cfg->V0 * (tau[3 * r] * gW[0] + tau[3 * r + 1] * gW[1] + tau[3 * r + 2] * gW[2]);
                }
    }
    return err;
}

/* G2P of the standard MPM (Sec. III-A): v_p = sum phi v_I and x += dt v_p
 * (Eq. 4), L = sum v_I grad phi^T and F = (I + dt L) F (Eq. 5), then the
 * plastic projection when enabled.  L is stored in C (the velocity gradient
 * the F update used; the standard P2G does not read it). */
int orc_g2p_standard(const orc_config* cfg, int N, double* x, double* v, double* C, double* F,
                     const double* mu, double dt, const double* gv)
{
    int err = 0, n = cfg->n;
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3], dw[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) bspline_w_dw(f[d], w[d], dw[d]);
        double vp[3] = {0, 0, 0}, L[9] = {0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double gW[3] = {n * dw[0][i] * w[1][j] * w[2][k], n * w[0][i] * dw[1][j] * w[2][k],
                                    n * w[0][i] * w[1][j] * dw[2][k]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    for (int r = 0; r < 3; ++r) {
                        vp[r] += W * gv[3 * I + r];
                        for (int c = 0; c < 3; ++c) L[3 * r + c] += gv[3 * I + r] * gW[c];
                    }
                }
        double G[9];
        for (int i = 0; i < 9; ++i) G[i] = ((i % 4 == 0) ? 1.0 : 0.0) + dt * L[i];
        matmul3(G, F + 9 * p, F + 9 * p);
        if (cfg->plasticity) err |= orc_von_mises(F + 9 * p, mu[p], cfg->yield_stress);
        for (int r = 0; r < 3; ++r) {
            v[3 * p + r] = vp[r];
            x[3 * p + r] += dt * vp[r];
        }
        memcpy(C + 9 * p, L, sizeof L);
        for (int i = 0; i < 3; ++i) if (!isfinite(x[3 * p + i]) || !isfinite(v[3 * p + i])) err |= ORC_ERR_NONFINITE;
        for (int i = 0; i < 9; ++i) if (!isfinite(F[9 * p + i])) err |= ORC_ERR_NONFINITE;
    }
    return err;
}

/* One substep of the standard MPM: P2G (Eq. 1, 2), the same node loop as
 * MLS-MPM (Eq. 3, contact, walls), G2P (Eq. 4, 5), reset, rigid advance and
 * push-out. */
int orc_substep_standard(const orc_config* cfg, int N, double* x, double* v, double* C, double* F,
                         const double* mu, const double* lam, int n_rigid, orc_rigid* rigids, double dt,
                         double* grid)
{
    int64_t nn = (int64_t)cfg->n * cfg->n * cfg->n;
    memset(grid, 0, (size_t)nn * 4 * sizeof(double));
    double* gm = grid;
    double* gmv = grid + nn;
    int err = orc_p2g_standard(cfg, N, x, v, F, mu, lam, dt, gm, gmv);
    if (err & ORC_ERR_OUT_OF_DOMAIN) return err;
    err |= orc_grid_update(cfg, gm, gmv, n_rigid, rigids, dt);
    err |= orc_g2p_standard(cfg, N, x, v, C, F, mu, dt, gmv);
    for (int r = 0; r < n_rigid; ++r) orc_rigid_advance(&rigids[r], dt);
    for (int p = 0; p < N; ++p)
        for (int r = 0; r < n_rigid; ++r) orc_push_out(&rigids[r], x + 3 * p);
    return err;
}

/* ------------------------------------------------------------- PB-MPM */

/* Co-rotational material constraint of PB-MPM (Sec. III-C), solved for one
 * particle: F* = (I + dt C) F, R from the polar decomposition of F*,
 * F* <- beta R + (1 - beta) F* / det(F*) (as printed), and the candidate
 * velocity gradient C <- (F* F^-1 - I) / dt.  Cout may alias C. */
void orc_pb_constraint(const double C[9], const double F[9], double dt, double beta, double Cout[9])
{
    double G[9], Fs[9], R[9], Finv[9], M[9];
    for (int i = 0; i < 9; ++i) G[i] = ((i % 4 == 0) ? 1.0 : 0.0) + dt * C[i];
    matmul3(G, F, Fs);
    orc_polar_R(Fs, R);
    double J = det3(Fs);
    for (int i = 0; i < 9; ++i) Fs[i] = beta * R[i] + (1.0 - beta) * Fs[i] / J;
    /* F^-1 by the adjugate */
    double dF = det3(F);
    Finv[0] = (F[4] * F[8] - F[5] * F[7]) / dF;
    Finv[1] = (F[2] * F[7] - F[1] * F[8]) / dF;
    Finv[2] = (F[1] * F[5] - F[2] * F[4]) / dF;
    Finv[3] = (F[5] * F[6] - F[3] * F[8]) / dF;
    Finv[4] = (F[0] * F[8] - F[2] * F[6]) / dF;
    Finv[5] = (F[2] * F[3] - F[0] * F[5]) / dF;
    Finv[6] = (F[3] * F[7] - F[4] * F[6]) / dF;
    Finv[7] = (F[1] * F[6] - F[0] * F[7]) / dF;
    Finv[8] = (F[0] * F[4] - F[1] * F[3]) / dF;
    matmul3(Fs, Finv, M);
    for (int i = 0; i < 9; ++i) Cout[i] = (M[i] - ((i % 4 == 0) ? 1.0 : 0.0)) / dt;
}

/* APIC P2G without a force term (the PB-MPM transfer): m_I += phi m (Eq. 1),
 * (m v)_I += phi m (v + C (x_I - x_p)). */
int orc_p2g_apic(const orc_config* cfg, int N, const double* x, const double* v, const double* C, double* gm,
                 double* gmv)
{
    int err = 0, n = cfg->n;
    double dx = 1.0 / n;
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) orc_bspline_weights(f[d], w[d]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double dpos[3] = {(b[0] + i) * dx - x[3 * p], (b[1] + j) * dx - x[3 * p + 1],
                                      (b[2] + k) * dx - x[3 * p + 2]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    gm[I] += W * cfg->m_p;
                    for (int r = 0; r < 3; ++r)
                        gmv[3 * I + r] += W * cfg->m_p * (v[3 * p + r] + C[9 * p + 3 * r] * dpos[0] +
                                                          C[9 * p + 3 * r + 1] * dpos[1] + C[9 * p + 3 * r + 2] * dpos[2]);
                }
    }
    return err;
}

/* G2P of one PB-MPM iteration: v_p = sum phi v_I (Eq. 4) and the APIC
 * C_p = (4/dx^2) sum phi v_I (x_I - x_p)^T (Eq. 9); positions and F wait for
 * the end of the step. */
int orc_g2p_vc(const orc_config* cfg, int N, const double* x, double* v, double* C, const double* gv)
{
    int err = 0, n = cfg->n;
    double dx = 1.0 / n, Dinv = 4.0 / (dx * dx);
    for (int p = 0; p < N; ++p) {
        int b[3];
        double f[3], w[3][3];
        int e = base_and_frac(cfg, x + 3 * p, b, f);
        if (e) { err |= e; continue; }
        for (int d = 0; d < 3; ++d) orc_bspline_weights(f[d], w[d]);
        double vp[3] = {0, 0, 0}, B[9] = {0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    double W = w[0][i] * w[1][j] * w[2][k];
                    double dpos[3] = {(b[0] + i) * dx - x[3 * p], (b[1] + j) * dx - x[3 * p + 1],
                                      (b[2] + k) * dx - x[3 * p + 2]};
                    int64_t I = ((int64_t)(b[0] + i) * n + (b[1] + j)) * n + (b[2] + k);
                    for (int r = 0; r < 3; ++r) {
                        vp[r] += W * gv[3 * I + r];
                        for (int c = 0; c < 3; ++c) B[3 * r + c] += W * gv[3 * I + r] * dpos[c];
                    }
                }
        for (int r = 0; r < 3; ++r) v[3 * p + r] = vp[r];
        for (int i = 0; i < 9; ++i) C[9 * p + i] = Dinv * B[i];
    }
    return err;
}

/* One PB-MPM step (Sec. III-C): `iters` P2G-G2P cycles at fixed positions,
 * each solving the co-rotational constraint of every particle in P2G (in
 * place of the stress), then the APIC transfer, the node loop and the APIC
 * G2P; then positions and F are integrated with the last velocity and
 * velocity gradient, the rigids advance and particles are pushed out.
 * Readings: gravity enters once per step (the first cycle's node loop; later
 * cycles start from velocities that already hold it); contact and walls act
 * in every cycle and every cycle's contact momentum is booked to the rigids. */
int orc_pb_step(const orc_config* cfg, int N, double* x, double* v, double* C, double* F, int n_rigid,
                orc_rigid* rigids, double dt, int iters, double beta, double* grid)
{
    int64_t nn = (int64_t)cfg->n * cfg->n * cfg->n;
    double* gm = grid;
    double* gmv = grid + nn;
    int err = 0;
    orc_config later = *cfg;
    later.gravity[0] = later.gravity[1] = later.gravity[2] = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int p = 0; p < N; ++p) orc_pb_constraint(C + 9 * p, F + 9 * p, dt, beta, C + 9 * p);
        memset(grid, 0, (size_t)nn * 4 * sizeof(double));
        err |= orc_p2g_apic(cfg, N, x, v, C, gm, gmv);
        if (err & ORC_ERR_OUT_OF_DOMAIN) return err;
        err |= orc_grid_update(it == 0 ? cfg : &later, gm, gmv, n_rigid, rigids, dt);
        err |= orc_g2p_vc(cfg, N, x, v, C, gmv);
    }
    for (int p = 0; p < N; ++p) {
        double G[9];
        for (int i = 0; i < 9; ++i) G[i] = ((i % 4 == 0) ? 1.0 : 0.0) + dt * C[9 * p + i];
        matmul3(G, F + 9 * p, F + 9 * p);
        for (int r = 0; r < 3; ++r) x[3 * p + r] += dt * v[3 * p + r];
        for (int i = 0; i < 3; ++i) if (!isfinite(x[3 * p + i]) || !isfinite(v[3 * p + i])) err |= ORC_ERR_NONFINITE;
        for (int i = 0; i < 9; ++i) if (!isfinite(F[9 * p + i])) err |= ORC_ERR_NONFINITE;
    }
    for (int r = 0; r < n_rigid; ++r) orc_rigid_advance(&rigids[r], dt);
    for (int p = 0; p < N; ++p)
        for (int r = 0; r < n_rigid; ++r) orc_push_out(&rigids[r], x + 3 * p);
    return err;
}

/* n_steps steps of a solver: 0 MLS-MPM (orc_substep), 1 standard MPM, 2
 * PB-MPM with `iters` cycles and stiffness beta.  Stops at the first error. */
int orc_run_solver(const orc_config* cfg, int solver, int N, double* x, double* v, double* C, double* F,
                   const double* mu, const double* lam, int n_rigid, orc_rigid* rigids, double dt, int n_steps,
                   int iters, double beta)
{
    int64_t nn = (int64_t)cfg->n * cfg->n * cfg->n;
    double* grid = (double*)malloc((size_t)nn * 4 * sizeof(double));
    if (!grid) return -1;
    int err = 0;
    for (int s = 0; s < n_steps && !err; ++s) {
        if (solver == 1) err = orc_substep_standard(cfg, N, x, v, C, F, mu, lam, n_rigid, rigids, dt, grid);
        else if (solver == 2) err = orc_pb_step(cfg, N, x, v, C, F, n_rigid, rigids, dt, iters, beta, grid);
        else err = orc_substep(cfg, N, x, v, C, F, mu, lam, n_rigid, rigids, dt, grid);
    }
    free(grid);
    return err;
}

/* ------------------------------------------------------------- binning */

/* Sort-by-cell: particles ordered by the 4^3-cell brick holding their base
 * cell, stable in the particle index.  The base cell is an integer decided by
 * floating point, so it is decided here in single precision as
 * floor(fma(x, n, -0.5)) (one rounding), clamped to [0, n-3]; brick key
 * ((bx*nb + by)*nb + bz) with nb = n/4.  Outputs: key[N], perm[N] (sorted
 * position -> particle), count[nb^3]. */
typedef struct { int key, idx; } orc_kv;

static int kv_cmp(const void* a, const void* b)
{
    const orc_kv* p = (const orc_kv*)a;
    const orc_kv* q = (const orc_kv*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

void orc_sort_by_brick(int n, int N, const float* x, int* key, int* perm, int* count)
{
    int nb = n / 4;
    memset(count, 0, sizeof(int) * (size_t)nb * nb * nb);
    orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(N > 0 ? N : 1));
    for (int p = 0; p < N; ++p) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            float s = floorf(fmaf(x[3 * p + d], (float)n, -0.5f));
            int b;
            if (!(s >= 0.0f)) b = 0; /* also NaN */
            else if (s > (float)(n - 3)) b = n - 3;
            else b = (int)s;
            c[d] = b / 4;
        }
        key[p] = (c[0] * nb + c[1]) * nb + c[2];
        count[key[p]]++;
        kv[p].key = key[p];
        kv[p].idx = p;
    }
    qsort(kv, (size_t)N, sizeof(orc_kv), kv_cmp);
    for (int s = 0; s < N; ++s) perm[s] = kv[s].idx;
    free(kv);
}

/* Trajectory loss of the differentiable workload: squared distance of the
 * particle centroid to a target plus the mean squared particle speed. */
double orc_loss(int N, const double* x, const double* v, const double target[3])
{
    double c[3] = {0, 0, 0}, kin = 0;
    for (int p = 0; p < N; ++p)
        for (int d = 0; d < 3; ++d) { c[d] += x[3 * p + d]; kin += v[3 * p + d] * v[3 * p + d]; }
    double l = 0;
    for (int d = 0; d < 3; ++d) { double e = c[d] / N - target[d]; l += e * e; }
    return l + kin / N;
}
