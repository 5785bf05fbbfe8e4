/*
 * fsi_oracle.c -- plain, slow, FP64 CPU restatement of the hot path of BIFROST's
 * fourth-order forward symplectic integrator (Rantala et al. 2022, arXiv 2210.02472).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked
 * against.  Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the CUDA
 * path, and it never reads anything the CUDA path computed.
 *
 * Every routine is a direct double loop over particle pairs in the order the paper's
 * equations are written, in FP64 with libm's correctly rounded sqrt.  There is no
 * blocking, no fusion and no reordering of the sums beyond the loop order stated.
 *
 * Layout: positions, velocities and accelerations are structure-of-arrays, 3 x N
 * doubles (all x, then all y, then all z).  Index lists are int32 global particle ids;
 * a NULL list means "all N particles in order".  Per-set outputs are 3 x n, in the
 * order of the index list.
 *
 * Pins (checked by the CPU test suite against closed forms, finite differences,
 * brute force and invariants): see the tests directory.  Every function here is pinned;
 * none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOMEM (-2)
#define OR_ERR_COINCIDENT (-4)
#define OR_ERR_MAXLEVEL (-6)
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------- */
static int or_threads = 1;

void or_set_threads(int n) { or_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return or_threads; }

static int idx_at(const int *list, int k) { return list ? list[k] : k; }

/* ------------------------------------------------------------------------------- *
 * Newtonian acceleration, Sect. 2.1 Eq. (new-newton-acc):
 *   a_i = sum_{j in B, j != i} G m_j r_ji / |r_ji|^3,  r_ji = r_j - r_i,  G = 1.
 * With Plummer softening |r_ji|^2 -> |r_ji|^2 + eps2.  Self pairs are excluded by
 * global index.  Two distinct particles at the same point with eps2 == 0 make the
 * sum undefined: the routine returns OR_ERR_COINCIDENT.
 * ------------------------------------------------------------------------------- */
int or_acc(int N, const double *pos, const double *mass,
           const int *A, int nA, const int *B, int nB, double eps2, double *acc)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < nA; ++k) {
        int i = idx_at(A, k);
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int l = 0; l < nB; ++l) {
            int j = idx_at(B, l);
            if (j == i) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double r = sqrt(r2);
            double f = mass[j] / (r2 * r);
            ax += f * dx;
            ay += f * dy;
            az += f * dz;
        }
        acc[k] = ax;
        acc[(size_t)nA + k] = ay;
        acc[2 * (size_t)nA + k] = az;
    }
    return err;
}

/* ------------------------------------------------------------------------------- *
 * Force-gradient sum of the gradient acceleration, Sect. 2.1 Eq. (new-grad-acc):
 *   G_i = sum_{j in B, j != i} G m_j / |r_ji|^5 ( |r_ji|^2 a_ji - 3 (a_ji . r_ji) r_ji ),
 *   a_ji = a_j - a_i,
 * so that the gradient acceleration is  a~_i = a_i + (eps^2 / 24) G_i.  The
 * accelerations are read from accg, a 3 x N array indexed by global particle id; the
 * caller fills it with the accelerations of the same splitting term (Sect. 2.2).
 * With softening, |r|^2 -> |r|^2 + eps2 in both powers (the exact softened Jacobian).
 * ------------------------------------------------------------------------------- */
int or_grad(int N, const double *pos, const double *mass, const double *accg,
            const int *A, int nA, const int *B, int nB, double eps2, double *grad)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *AX = accg, *AY = accg + N, *AZ = accg + 2 * (size_t)N;
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < nA; ++k) {
        int i = idx_at(A, k);
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int l = 0; l < nB; ++l) {
            int j = idx_at(B, l);
            if (j == i) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double bx = AX[j] - AX[i], by = AY[j] - AY[i], bz = AZ[j] - AZ[i];
            double r = sqrt(r2);
            double r5 = r2 * r2 * r;
            double f = mass[j] / r5;
            double adotr = bx * dx + by * dy + bz * dz;
            gx += f * (r2 * bx - 3.0 * adotr * dx);
            gy += f * (r2 * by - 3.0 * adotr * dy);
            gz += f * (r2 * bz - 3.0 * adotr * dz);
        }
        grad[k] = gx;
        grad[(size_t)nA + k] = gy;
        grad[2 * (size_t)nA + k] = gz;
    }
    return err;
}

/* 1 if the two lists hold the same ids in the same order, 0 if they share no id,
 * -1 otherwise (partial overlap has no meaning for a splitting term). */
static int classify_sets(int N, const int *A, int nA, const int *B, int nB)
{
    if (nA == nB) {
        int same = 1;
        for (int k = 0; k < nA; ++k)
            if (idx_at(A, k) != idx_at(B, k)) { same = 0; break; }
        if (same) return 1;
    }
    unsigned char *mark = (unsigned char *)calloc((size_t)N, 1);
    if (!mark) return -2;
    for (int k = 0; k < nA; ++k) mark[idx_at(A, k)] = 1;
    int overlap = 0;
    for (int l = 0; l < nB; ++l)
        if (mark[idx_at(B, l)]) { overlap = 1; break; }
    free(mark);
    return overlap ? -1 : 0;
}

/* Scatter a 3 x n per-set array into a 3 x N global-id array. */
static void scatter3(int N, const int *list, int n, const double *src, double *dstg)
{
    for (int k = 0; k < n; ++k) {
        int i = idx_at(list, k);
        dstg[i] = src[k];
        dstg[(size_t)N + i] = src[(size_t)n + k];
        dstg[2 * (size_t)N + i] = src[2 * (size_t)n + k];
    }
}

/* ------------------------------------------------------------------------------- *
 * acc(A <- B) and the gradient sum G(A <- B) of one splitting term.
 *  - A and B the same list: the term is the set's self-interaction (FSI, Sect. 2.1);
 *    the accelerations inside G are acc(A <- A).
 *  - A and B disjoint: the term is the slow-fast inter-level interaction (Sect. 2.2);
 *    a_i = acc(A <- B) for i in A and a_j = acc(B <- A) for j in B.
 * Any other overlap is rejected with OR_ERR_ARG.
 * ------------------------------------------------------------------------------- */
int or_accel_grad(int N, const double *pos, const double *mass,
                  const int *A, int nA, const int *B, int nB, double eps2,
                  double *acc_out, double *grad_out)
{
    int kind = classify_sets(N, A, nA, B, nB);
    if (kind == -2) return OR_ERR_NOMEM;
    if (kind < 0) return OR_ERR_ARG;
    double *accg = (double *)calloc(3 * (size_t)N, sizeof(double));
    double *tmp = (double *)malloc(3 * (size_t)(nB > 0 ? nB : 1) * sizeof(double));
    if (!accg || !tmp) { free(accg); free(tmp); return OR_ERR_NOMEM; }
    int err = or_acc(N, pos, mass, A, nA, B, nB, eps2, acc_out);
    scatter3(N, A, nA, acc_out, accg);
    if (kind == 0 && err == OR_OK) {
        err = or_acc(N, pos, mass, B, nB, A, nA, eps2, tmp);
        scatter3(N, B, nB, tmp, accg);
    }
    if (err == OR_OK)
        err = or_grad(N, pos, mass, accg, A, nA, B, nB, eps2, grad_out);
    free(accg);
    free(tmp);
    return err;
}

/* ------------------------------------------------------------------------------- *
 * PN1.0 pair acceleration (Sect. 3.9, Eqs. subsyspn-mass and the FSI+PN splitting).
 * The paper does not print the pair formula; it takes the PN terms of Thorne (1985)
 * and the Einstein-Infeld-Hoffmann equations restricted to pairs.  The two-body 1PN
 * EIH acceleration of body i due to body j in harmonic coordinates, with
 * n = (x_i - x_j)/r, is
 *   a_i = (G m_j / (c^2 r^2)) { n [ -v_i^2 - 2 v_j^2 + 4 v_i.v_j + 3/2 (n.v_j)^2
 *                                   + 5 G m_i / r + 4 G m_j / r ]
 *                               + (v_i - v_j) [ 4 n.v_i - 3 n.v_j ] }.
 * A pair contributes only when at least one member is flagged as a black hole (the
 * mass cut of Eq. subsyspn-mass, read as m > m_PN).  No softening is applied.
 * For i in A the sum runs over j in B, j != i.
 * ------------------------------------------------------------------------------- */
int or_pn_acc(int N, const double *pos, const double *vel, const double *mass,
              const unsigned char *is_bh, double c,
              const int *A, int nA, const int *B, int nB, double *out)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *VX = vel, *VY = vel + N, *VZ = vel + 2 * (size_t)N;
    double ic2 = 1.0 / (c * c);
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < nA; ++k) {
        int i = idx_at(A, k);
        double px = 0.0, py = 0.0, pz = 0.0;
        for (int l = 0; l < nB; ++l) {
            int j = idx_at(B, l);
            if (j == i) continue;
            if (!is_bh[i] && !is_bh[j]) continue;
            double rx = X[i] - X[j], ry = Y[i] - Y[j], rz = Z[i] - Z[j];
            double r = sqrt(rx * rx + ry * ry + rz * rz);
            if (r == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double nx = rx / r, ny = ry / r, nz = rz / r;
            double vi2 = VX[i] * VX[i] + VY[i] * VY[i] + VZ[i] * VZ[i];
            double vj2 = VX[j] * VX[j] + VY[j] * VY[j] + VZ[j] * VZ[j];
            double vivj = VX[i] * VX[j] + VY[i] * VY[j] + VZ[i] * VZ[j];
            double nvi = nx * VX[i] + ny * VY[i] + nz * VZ[i];
            double nvj = nx * VX[j] + ny * VY[j] + nz * VZ[j];
            double cn = -vi2 - 2.0 * vj2 + 4.0 * vivj + 1.5 * nvj * nvj
                        + 5.0 * mass[i] / r + 4.0 * mass[j] / r;
            double cv = 4.0 * nvi - 3.0 * nvj;
            double pre = mass[j] * ic2 / (r * r);
            px += pre * (cn * nx + cv * (VX[i] - VX[j]));
            py += pre * (cn * ny + cv * (VY[i] - VY[j]));
            pz += pre * (cn * nz + cv * (VZ[i] - VZ[j]));
        }
        out[k] = px;
        out[(size_t)nA + k] = py;
        out[2 * (size_t)nA + k] = pz;
    }
    return err;
}

/* ------------------------------------------------------------------------------- *
 * Energy, Sect. 2.1 (the Hamiltonian):
 *   T = sum_i 1/2 m_i |v_i|^2,  W = - sum_{i<j} G m_i m_j / sqrt(|r_ij|^2 + eps2),
 * over the listed set.
 * ------------------------------------------------------------------------------- */
int or_energy(int N, const double *pos, const double *vel, const double *mass,
              const int *P, int n, double eps2, double *ekin, double *epot)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *VX = vel, *VY = vel + N, *VZ = vel + 2 * (size_t)N;
    double t = 0.0, w = 0.0;
    int err = OR_OK;
    for (int k = 0; k < n; ++k) {
        int i = idx_at(P, k);
        t += 0.5 * mass[i] * (VX[i] * VX[i] + VY[i] * VY[i] + VZ[i] * VZ[i]);
    }
    int k;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : w) num_threads(or_threads)
    for (k = 0; k < n; ++k) {
        int i = idx_at(P, k);
        for (int l = k + 1; l < n; ++l) {
            int j = idx_at(P, l);
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            w -= mass[i] * mass[j] / sqrt(r2);
        }
    }
    *ekin = t;
    *epot = w;
    return err;
}

/* ------------------------------------------------------------------------------- */
typedef struct {
    double eps2;
    double c;                    /* speed of light; 0 switches the PN1.0 term off */
    const unsigned char *is_bh;  /* black-hole flags, N entries (may be NULL if c == 0) */
} or_force_params;

static void kick(int N, double *vel, const int *P, int n, const double *a, double w)
{
    for (int k = 0; k < n; ++k) {
        int i = idx_at(P, k);
        vel[i] += w * a[k];
        vel[(size_t)N + i] += w * a[(size_t)n + k];
        vel[2 * (size_t)N + i] += w * a[2 * (size_t)n + k];
    }
}

static void drift(int N, double *pos, const double *vel, const int *P, int n, double w)
{
    for (int k = 0; k < n; ++k) {
        int i = idx_at(P, k);
        pos[i] += w * vel[i];
        pos[(size_t)N + i] += w * vel[(size_t)N + i];
        pos[2 * (size_t)N + i] += w * vel[2 * (size_t)N + i];
    }
}

/* PN1.0 kick of the pairs (A x B), both directions for disjoint sets: all PN
 * accelerations are evaluated from the velocities at the start of the kick, then
 * applied (Sect. 3.9, the half-kicks that wrap the FSI). */
static int pn_kick(int N, const double *pos, double *vel, const double *mass,
                   const or_force_params *fp, const int *A, int nA,
                   const int *B, int nB, int same, double w)
{
    if (fp == NULL || fp->c <= 0.0 || w == 0.0) return OR_OK;
    double *aA = (double *)malloc(3 * (size_t)(nA > 0 ? nA : 1) * sizeof(double));
    double *aB = (double *)malloc(3 * (size_t)(nB > 0 ? nB : 1) * sizeof(double));
    if (!aA || !aB) { free(aA); free(aB); return OR_ERR_NOMEM; }
    int err = or_pn_acc(N, pos, vel, mass, fp->is_bh, fp->c, A, nA, B, nB, aA);
    if (!same && err == OR_OK)
        err = or_pn_acc(N, pos, vel, mass, fp->is_bh, fp->c, B, nB, A, nA, aB);
    if (err == OR_OK) {
        kick(N, vel, A, nA, aA, w);
        if (!same) kick(N, vel, B, nB, aB, w);
    }
    free(aA);
    free(aB);
    return err;
}

/* ------------------------------------------------------------------------------- *
 * Kick then drift of the listed set with given accelerations (the kinetic and potential
 * factors of Eq. fsi-cycle applied on their own): for k < n, i = P[k] (P NULL: i = k),
 *   v_i <- v_i + c_kick a_k,   then   x_i <- x_i + c_drift v_i.
 * acc: 3 x n compact rows (NULL: drift only).
 * ------------------------------------------------------------------------------- */
int or_kick_drift(int N, double *pos, double *vel, const double *acc, const int *P, int n,
                  double c_kick, double c_drift) {
    if (N < 0 || n < 0 || (!P && n > N)) return OR_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        const int i = P ? P[k] : k;
        if (i < 0 || i >= N) return OR_ERR_ARG;
        for (int c = 0; c < 3; ++c) {
            double v = vel[(size_t)c * N + i];
            if (acc) v = v + c_kick * acc[(size_t)c * n + k];
            vel[(size_t)c * N + i] = v;
            pos[(size_t)c * N + i] = pos[(size_t)c * N + i] + c_drift * v;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------- *
 * One FSI cycle of step h on the listed set, interacting with itself only
 * (Sect. 2.1, Eq. fsi-cycle):
 *   kick h/6 with a;  drift h/2;  kick 2h/3 with a~ = a + (h^2/24) G;  drift h/2;
 *   kick h/6 with a,
 * every acceleration evaluated at the current positions.  With the PN1.0 term on,
 * PN half-kicks of h/2 wrap the cycle (Sect. 3.9).
 * ------------------------------------------------------------------------------- */
int or_fsi_step(int N, double *pos, double *vel, const double *mass,
                const int *P, int n, double h, const or_force_params *fp)
{
    if (n <= 0) return OR_OK;
    double eps2 = fp ? fp->eps2 : 0.0;
    double *a = (double *)malloc(3 * (size_t)n * sizeof(double));
    double *g = (double *)malloc(3 * (size_t)n * sizeof(double));
    double *a3 = (double *)malloc(3 * (size_t)n * sizeof(double));
    if (!a || !g || !a3) { free(a); free(g); free(a3); return OR_ERR_NOMEM; }
    int err = pn_kick(N, pos, vel, mass, fp, P, n, P, n, 1, 0.5 * h);
    if (err == OR_OK) err = or_acc(N, pos, mass, P, n, P, n, eps2, a);
    if (err == OR_OK) {
        kick(N, vel, P, n, a, h / 6.0);
        drift(N, pos, vel, P, n, 0.5 * h);
        err = or_accel_grad(N, pos, mass, P, n, P, n, eps2, a, g);
    }
    if (err == OR_OK) {
        for (size_t q = 0; q < 3 * (size_t)n; ++q) a3[q] = a[q] + (h * h / 24.0) * g[q];
        kick(N, vel, P, n, a3, 2.0 * h / 3.0);
        drift(N, pos, vel, P, n, 0.5 * h);
        err = or_acc(N, pos, mass, P, n, P, n, eps2, a);
    }
    if (err == OR_OK) {
        kick(N, vel, P, n, a, h / 6.0);
        err = pn_kick(N, pos, vel, mass, fp, P, n, P, n, 1, 0.5 * h);
    }
    free(a);
    free(g);
    free(a3);
    return err;
}

/* =============================================================================== *
 * FSI with subsystems (Sect. 2.3, Algorithm 1), kernel side: the splitting
 * H = T' + U' + sum_s H_S^s with U' = U minus the intra-subsystem potentials.  The kicks
 * use accelerations and gradient sums that ignore every pair inside one subsystem; the
 * drifts move only the single particles; each subsystem is advanced by its own
 * Hamiltonian H_S (its members' kinetic energy plus their mutual potential) for eps/2
 * twice per cycle.  Subsystems here are isolated bound binaries, whose H_S flow is the
 * exact two-body (Kepler) motion: the centre of mass moves on a straight line and the
 * relative orbit follows Kepler's equation (Sect. 3.11).
 * sub[i] (N entries, global id) is the subsystem of particle i, -1 for a single.
 * =============================================================================== */
static int same_subsystem(const int *sub, int i, int j)
{
    return sub && sub[i] >= 0 && sub[i] == sub[j];
}

/* acc(A <- B) without intra-subsystem pairs (plain definition, as or_acc). */
int or_acc_sub(int N, const double *pos, const double *mass, const int *sub,
               const int *A, int nA, const int *B, int nB, double eps2, double *acc)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < nA; ++k) {
        int i = idx_at(A, k);
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int l = 0; l < nB; ++l) {
            int j = idx_at(B, l);
            if (j == i || same_subsystem(sub, i, j)) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double f = mass[j] / (r2 * sqrt(r2));
            ax += f * dx; ay += f * dy; az += f * dz;
        }
        acc[k] = ax;
        acc[(size_t)nA + k] = ay;
        acc[2 * (size_t)nA + k] = az;
    }
    return err;
}

/* grad(A <- B) without intra-subsystem pairs; accg is a 3 x N global-id field. */
int or_grad_sub(int N, const double *pos, const double *mass, const int *sub,
                const double *accg, const int *A, int nA, const int *B, int nB, double eps2,
                double *grad)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *AX = accg, *AY = accg + N, *AZ = accg + 2 * (size_t)N;
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < nA; ++k) {
        int i = idx_at(A, k);
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int l = 0; l < nB; ++l) {
            int j = idx_at(B, l);
            if (j == i || same_subsystem(sub, i, j)) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double bx = AX[j] - AX[i], by = AY[j] - AY[i], bz = AZ[j] - AZ[i];
            double r = sqrt(r2);
            double f = mass[j] / (r2 * r2 * r);
            double adotr = bx * dx + by * dy + bz * dz;
            gx += f * (r2 * bx - 3.0 * adotr * dx);
            gy += f * (r2 * by - 3.0 * adotr * dy);
            gz += f * (r2 * bz - 3.0 * adotr * dz);
        }
        grad[k] = gx;
        grad[(size_t)nA + k] = gy;
        grad[2 * (size_t)nA + k] = gz;
    }
    return err;
}

/* Kepler's equation M = E - e sin E (Sect. 3.11): the cubic first approximation in
 * s = sin(E/3) (arcsin expanded to third order; the real root of
 * (1 - e) s + (1/6 + 4e/3) s^3 = M/3), then Newton-Raphson with a bisection fallback,
 * until two consecutive iterates differ by less than tol. */
static double kepler_solve(double M, double e, double tol)
{
    double twopi = 2.0 * OR_PI;
    double k = floor((M + OR_PI) / twopi);
    double Mr = M - k * twopi;
    double sgn = Mr >= 0.0 ? 1.0 : -1.0;
    double Ma = fabs(Mr);
    double c3 = 1.0 / 6.0 + 4.0 * e / 3.0;
    double p = (1.0 - e) / c3, q = (Ma / 3.0) / c3;
    double s;
    if (p > 0.0) {
        double al = 2.0 * sqrt(p / 3.0);
        s = al * sinh(asinh(4.0 * q / (al * al * al)) / 3.0);
    } else {
        s = cbrt(q);
    }
    if (s > 1.0) s = 1.0;
    double E = 3.0 * asin(s);
    double lo = 0.0, hi = OR_PI;
    for (int it = 0; it < 200; ++it) {
        double f = E - e * sin(E) - Ma;
        if (f > 0.0) { if (E < hi) hi = E; }
        else if (E > lo) lo = E;
        double En = E - f / (1.0 - e * cos(E));
        if (!(En >= lo && En <= hi)) En = 0.5 * (lo + hi);
        double d = fabs(En - E);
        E = En;
        if (d < tol) break;
    }
    return sgn * E + k * twopi;
}

/* Exact two-body motion of particles i, j over time t (bound orbits only). */
static int kepler_drift(int N, double *pos, double *vel, const double *mass, int i, int j,
                        double t)
{
    double mi = mass[i], mj = mass[j], mu = mi + mj;
    double R[3], V[3], r0[3], v0[3];
    for (int q = 0; q < 3; ++q) {
        size_t oi = (size_t)q * N + i, oj = (size_t)q * N + j;
        R[q] = (mi * pos[oi] + mj * pos[oj]) / mu;
        V[q] = (mi * vel[oi] + mj * vel[oj]) / mu;
        r0[q] = pos[oj] - pos[oi];
        v0[q] = vel[oj] - vel[oi];
    }
    double r0n = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    double v02 = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
    double rv = r0[0] * v0[0] + r0[1] * v0[1] + r0[2] * v0[2];
    double inva = 2.0 / r0n - v02 / mu;
    if (!(inva > 0.0)) return OR_ERR_ARG;           /* unbound: not a binary */
    double a = 1.0 / inva;
    double n = sqrt(mu * inva * inva * inva);
    double ec = 1.0 - r0n / a;                      /* e cos E0 */
    double es = rv / sqrt(mu * a);                  /* e sin E0 */
    double e = sqrt(ec * ec + es * es);
    double E0 = atan2(es, ec);
    double M0 = E0 - es;
    double E1 = kepler_solve(M0 + n * t, e, 1e-15);
    double dE = E1 - E0;
    double f = 1.0 - (a / r0n) * (1.0 - cos(dE));
    double g = t - (dE - sin(dE)) / n;
    double r1[3];
    for (int q = 0; q < 3; ++q) r1[q] = f * r0[q] + g * v0[q];
    double r1n = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    double fd = -sqrt(mu * a) * sin(dE) / (r0n * r1n);
    double gd = 1.0 - (a / r1n) * (1.0 - cos(dE));
    for (int q = 0; q < 3; ++q) {
        double v1 = fd * r0[q] + gd * v0[q];
        double Rq = R[q] + V[q] * t;
        size_t oi = (size_t)q * N + i, oj = (size_t)q * N + j;
        pos[oi] = Rq - (mj / mu) * r1[q];
        pos[oj] = Rq + (mi / mu) * r1[q];
        vel[oi] = V[q] - (mj / mu) * v1;
        vel[oj] = V[q] + (mi / mu) * v1;
    }
    return OR_OK;
}

/* One FSI cycle of set P with the binary subsystems listed in pairs (n_pairs pairs of
 * global ids, members of P; sub must mark them: sub[pairs[2s]] = sub[pairs[2s+1]] = s and
 * -1 for every other particle), Algorithm 1:
 *   kick eps/6 (a'), subsystems eps/2, drift singles eps/2, kick 2eps/3 (a' + eps^2/24 G'),
 *   subsystems eps/2, drift singles eps/2, kick eps/6 (a'),
 * where a' and G' ignore the intra-subsystem pairs (G' from the a' of the same term). */
int or_fsi_step_sub(int N, double *pos, double *vel, const double *mass, const int *sub,
                    const int *pairs, int n_pairs, const int *P, int n, double h, double eps2)
{
    if (n <= 0) return OR_OK;
    double *a = (double *)malloc(3 * (size_t)n * sizeof(double));
    double *g = (double *)malloc(3 * (size_t)n * sizeof(double));
    double *field = (double *)calloc(3 * (size_t)N, sizeof(double));
    if (!a || !g || !field) { free(a); free(g); free(field); return OR_ERR_NOMEM; }
    int err = OR_OK;
    for (int half = 0; half < 2 && err == OR_OK; ++half) {
        /* opening kick eps/6 (half 0) or gradient kick 2 eps/3 (half 1) */
        err = or_acc_sub(N, pos, mass, sub, P, n, P, n, eps2, a);
        if (err == OR_OK && half == 1) {
            for (int k = 0; k < n; ++k)
                for (int q = 0; q < 3; ++q) field[(size_t)q * N + idx_at(P, k)] = a[(size_t)q * n + k];
            err = or_grad_sub(N, pos, mass, sub, field, P, n, P, n, eps2, g);
            if (err == OR_OK)
                for (size_t q = 0; q < 3 * (size_t)n; ++q) a[q] += (h * h / 24.0) * g[q];
        }
        if (err != OR_OK) break;
        kick(N, vel, P, n, a, half == 0 ? h / 6.0 : 2.0 * h / 3.0);
        for (int s = 0; s < n_pairs && err == OR_OK; ++s)
            err = kepler_drift(N, pos, vel, mass, pairs[2 * s], pairs[2 * s + 1], 0.5 * h);
        for (int k = 0; k < n && err == OR_OK; ++k) {
            int i = idx_at(P, k);
            if (sub[i] >= 0) continue;
            for (int q = 0; q < 3; ++q) pos[(size_t)q * N + i] += 0.5 * h * vel[(size_t)q * N + i];
        }
    }
    if (err == OR_OK) err = or_acc_sub(N, pos, mass, sub, P, n, P, n, eps2, a);
    if (err == OR_OK) kick(N, vel, P, n, a, h / 6.0);
    free(a);
    free(g);
    free(field);
    return err;
}

/* Time-step parameters (Sect. 3.4): eta_grad and eta_va switch their criteria off at 0. */
typedef struct {
    double eta_ff, eta_fb, eta_jerk, eta_grad, eta_va;
} or_step_params;

/* ------------------------------------------------------------------------------- *
 * Time steps of the listed set against itself (Sect. 3.4):
 *   free fall  eps_ff = eta_ff min_{j != i} ( |r_ij|^3 / (G (m_i + m_j)) )^{1/2},
 *   fly-by     eps_fb = eta_fb min_{j != i} |r_ij| / |v_ij|,
 *   jerk       eps_j  = eta_j |a_i| / |j_i|,
 *              j_i = sum_{j != i} G m_j / |r_ji|^5 ( |r_ji|^2 v_ji - 3 (r_ji . v_ji) r_ji ),
 * the step being the minimum of the three.  A pair at zero relative speed gives no
 * fly-by bound and a zero jerk gives no jerk bound (both +inf).  The free-fall and
 * fly-by distances are unsoftened; a_i and j_i use the softened kernel of the force.
 * ------------------------------------------------------------------------------- */
static int steps_ff_fb_jerk(int N, const double *pos, const double *vel,
                            const double *mass, const int *P, int n, double eta_ff,
                            double eta_fb, double eta_jerk, double eps2, double *step,
                            double *acc)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *VX = vel, *VY = vel + N, *VZ = vel + 2 * (size_t)N;
    int err = OR_OK;
    int k;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (k = 0; k < n; ++k) {
        int i = idx_at(P, k);
        double ff2 = INFINITY, fb = INFINITY;
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
        for (int l = 0; l < n; ++l) {
            int j = idx_at(P, l);
            if (j == i) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double ux = VX[j] - VX[i], uy = VY[j] - VY[i], uz = VZ[j] - VZ[i];
            double d2 = dx * dx + dy * dy + dz * dz;
            double s2 = d2 + eps2;
            if (s2 == 0.0 || d2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double d = sqrt(d2);
            double t2 = d2 * d / (mass[i] + mass[j]);
            if (t2 < ff2) ff2 = t2;
            double u2 = ux * ux + uy * uy + uz * uz;
            if (u2 > 0.0) {
                double t = d / sqrt(u2);
                if (t < fb) fb = t;
            }
            double s = sqrt(s2);
            double f3 = mass[j] / (s2 * s);
            double f5 = f3 / s2;
            double rv = dx * ux + dy * uy + dz * uz;
            ax += f3 * dx; ay += f3 * dy; az += f3 * dz;
            jx += f5 * (s2 * ux - 3.0 * rv * dx);
            jy += f5 * (s2 * uy - 3.0 * rv * dy);
            jz += f5 * (s2 * uz - 3.0 * rv * dz);
        }
        double e = eta_ff * sqrt(ff2);
        double efb = eta_fb * fb;
        if (efb < e) e = efb;
        double jn = sqrt(jx * jx + jy * jy + jz * jz);
        if (jn > 0.0) {
            double ej = eta_jerk * sqrt(ax * ax + ay * ay + az * az) / jn;
            if (ej < e) e = ej;
        }
        step[k] = e;
        if (acc) {
            acc[k] = ax;
            acc[(size_t)n + k] = ay;
            acc[2 * (size_t)n + k] = az;
        }
    }
    return err;
}

int or_timesteps(int N, const double *pos, const double *vel, const double *mass,
                 const int *P, int n, double eta_ff, double eta_fb, double eta_jerk,
                 double eps2, double *step)
{
    return steps_ff_fb_jerk(N, pos, vel, mass, P, n, eta_ff, eta_fb, eta_jerk, eps2, step,
                            NULL);
}

/* ------------------------------------------------------------------------------- *
 * Every time-step criterion of Sect. 3.4 for the listed set against itself: the free-fall,
 * fly-by and jerk steps above, then, when switched on (parameter > 0),
 *   velocity per acceleration (Eq. vel-acc-crit)   eps = eta_va |v_i| / |a_i|,
 *   gradient, first form      (Eq. dt-nabla1)      eps = eta_grad (|v_i| / |g'_i|)^{1/3},
 *   gradient, second form     (Eq. dt-nabla2)      eps = eta_grad (|a_i| / |g'_i|)^{1/2},
 * where a_i is the acceleration from the set, g'_i the gradient acceleration of the FSI
 * gradient kick written as a~_i = a_i + eps^2 g'_i, i.e. g'_i = G_i / 24 with G_i the
 * force-gradient sum of Eq. new-grad-acc evaluated with the set's own accelerations, and
 * v_i the particle's velocity in the simulation frame.  |a_i| = 0 gives no
 * velocity-per-acceleration bound and |g'_i| = 0 no gradient bound.  The step is the
 * minimum over the criteria in use.
 * ------------------------------------------------------------------------------- */
int or_timesteps_all(int N, const double *pos, const double *vel, const double *mass,
                     const int *P, int n, const or_step_params *sp, double eps2, double *step)
{
    int extra = sp->eta_grad > 0.0 || sp->eta_va > 0.0;
    double *a = NULL, *field = NULL, *G = NULL;
    if (extra) {
        a = (double *)malloc(3 * (size_t)n * sizeof(double));
        field = (double *)calloc(3 * (size_t)N, sizeof(double));
        G = (double *)malloc(3 * (size_t)n * sizeof(double));
        if (!a || !field || !G) { free(a); free(field); free(G); return OR_ERR_NOMEM; }
    }
    int err = steps_ff_fb_jerk(N, pos, vel, mass, P, n, sp->eta_ff, sp->eta_fb, sp->eta_jerk,
                               eps2, step, a);
    if (err == OR_OK && extra) {
        /* the set's accelerations as a global-id field, then G_i from those (Sect. 2.1) */
        for (int k = 0; k < n; ++k) {
            int i = idx_at(P, k);
            for (int q = 0; q < 3; ++q) field[(size_t)q * N + i] = a[(size_t)q * n + k];
        }
        err = or_grad(N, pos, mass, field, P, n, P, n, eps2, G);
    }
    if (err == OR_OK && extra) {
        for (int k = 0; k < n; ++k) {
            int i = idx_at(P, k);
            double an = 0.0, gn = 0.0, vn = 0.0;
            for (int q = 0; q < 3; ++q) {
                double aq = a[(size_t)q * n + k], gq = G[(size_t)q * n + k] / 24.0;
                double vq = vel[(size_t)q * N + i];
                an += aq * aq;
                gn += gq * gq;
                vn += vq * vq;
            }
            an = sqrt(an);
            gn = sqrt(gn);
            vn = sqrt(vn);
            double e = step[k];
            if (sp->eta_va > 0.0 && an > 0.0) {
                double t = sp->eta_va * vn / an;
                if (t < e) e = t;
            }
            if (sp->eta_grad > 0.0 && gn > 0.0) {
                double t1 = sp->eta_grad * cbrt(vn / gn);
                double t2 = sp->eta_grad * sqrt(an / gn);
                if (t1 < e) e = t1;
                if (t2 < e) e = t2;
            }
            step[k] = e;
        }
    }
    free(a);
    free(field);
    free(G);
    return err;
}

/* ------------------------------------------------------------------------------- *
 * Hierarchical Hamiltonian splitting with the FSI (Sect. 2.2, Eq. hhsfsi-cycle),
 * literal reading: a level of pivot tau over set P
 *   1. assigns time steps against P (level 0: against all N, stored as the level-0
 *      steps; deeper levels take min(eps_i, eps_i^{level 0}), Sect. 3.4),
 *   2. splits S = {eps_i >= tau}, F = {eps_i < tau} (at max_level, S = P),
 *   3. runs  U_SF(tau/6)  FSI(S, tau/2)  HHS(F, tau/2)  U~_SF(2 tau/3)  HHS(F, tau/2)
 *            FSI(S, tau/2)  U_SF(tau/6),
 *      where U_SF kicks S with acc(S <- F) and F with acc(F <- S), and U~_SF uses the
 *      gradient accelerations of the same inter-level term with eps = tau.
 * With the PN1.0 term on, S-S pairs get the half-kicks that wrap each FSI(S, .) and
 * S-F pairs get PN kicks of tau/2 together with the opening and closing U_SF.
 * ------------------------------------------------------------------------------- */
typedef struct {
    double eta_ff, eta_fb, eta_jerk;
    double eps2;
    double c;
    const unsigned char *is_bh;
    int max_level;
    const double *fixed_steps;   /* if non-NULL: eps_i = fixed_steps[i] at every level */
    double eta_grad, eta_va;     /* gradient and velocity/acceleration criteria (0 = off) */
} or_hhs_params;

static or_step_params hhs_step_params(const or_hhs_params *p)
{
    or_step_params sp = {p->eta_ff, p->eta_fb, p->eta_jerk, p->eta_grad, p->eta_va};
    return sp;
}

typedef struct {
    int N;
    double *pos, *vel;
    const double *mass;
    const or_hhs_params *p;
    double *step0;        /* level-0 steps, global id */
    long long *level_counts;
    int max_level_hit;
} hhs_ctx;

static int cross_kick(hhs_ctx *c, const int *S, int nS, const int *F, int nF,
                      double w, int gradient, double eps)
{
    int N = c->N;
    double *aS = (double *)malloc(3 * (size_t)nS * sizeof(double));
    double *aF = (double *)malloc(3 * (size_t)nF * sizeof(double));
    double *gS = (double *)malloc(3 * (size_t)nS * sizeof(double));
    double *gF = (double *)malloc(3 * (size_t)nF * sizeof(double));
    if (!aS || !aF || !gS || !gF) {
        free(aS); free(aF); free(gS); free(gF);
        return OR_ERR_NOMEM;
    }
    int err;
    if (!gradient) {
        err = or_acc(N, c->pos, c->mass, S, nS, F, nF, c->p->eps2, aS);
        if (err == OR_OK) err = or_acc(N, c->pos, c->mass, F, nF, S, nS, c->p->eps2, aF);
    } else {
        err = or_accel_grad(N, c->pos, c->mass, S, nS, F, nF, c->p->eps2, aS, gS);
        if (err == OR_OK)
            err = or_accel_grad(N, c->pos, c->mass, F, nF, S, nS, c->p->eps2, aF, gF);
        if (err == OR_OK) {
            double f = eps * eps / 24.0;
            for (size_t q = 0; q < 3 * (size_t)nS; ++q) aS[q] += f * gS[q];
            for (size_t q = 0; q < 3 * (size_t)nF; ++q) aF[q] += f * gF[q];
        }
    }
    if (err == OR_OK) {
        kick(N, c->vel, S, nS, aS, w);
        kick(N, c->vel, F, nF, aF, w);
    }
    free(aS); free(aF); free(gS); free(gF);
    return err;
}

static int hhs_level(hhs_ctx *c, const int *P, int n, double tau, int level)
{
    int N = c->N;
    const or_hhs_params *p = c->p;
    if (n <= 0) return OR_OK;
    double *st = (double *)malloc((size_t)n * sizeof(double));
    int *S = (int *)malloc((size_t)n * sizeof(int));
    int *F = (int *)malloc((size_t)n * sizeof(int));
    if (!st || !S || !F) { free(st); free(S); free(F); return OR_ERR_NOMEM; }
    int err = OR_OK;
    if (p->fixed_steps)
        for (int k = 0; k < n; ++k) st[k] = p->fixed_steps[P[k]];
    else {
        or_step_params sp = hhs_step_params(p);
        err = or_timesteps_all(N, c->pos, c->vel, c->mass, P, n, &sp, p->eps2, st);
    }
    int nS = 0, nF = 0;
    if (err == OR_OK) {
        for (int k = 0; k < n; ++k) {
            int i = P[k];
            double e = st[k];
            if (level == 0) c->step0[i] = e;
            else if (c->step0[i] < e) e = c->step0[i];
            if (level >= p->max_level || e >= tau) S[nS++] = i;
            else F[nF++] = i;
        }
        if (level >= p->max_level && nS > 0 && n > 0) {
            /* count particles that wanted a smaller step than the deepest level allows */
            for (int k = 0; k < n; ++k) {
                double e = st[k];
                if (c->step0[P[k]] < e) e = c->step0[P[k]];
                if (e < tau) { c->max_level_hit = 1; break; }
            }
        }
        if (c->level_counts) c->level_counts[level] += nS;
    }
    or_force_params fp = {p->eps2, p->c, p->is_bh};
    int cross = (nS > 0 && nF > 0);
    if (err == OR_OK && cross) {
        err = pn_kick(N, c->pos, c->vel, c->mass, &fp, S, nS, F, nF, 0, 0.5 * tau);
        if (err == OR_OK) err = cross_kick(c, S, nS, F, nF, tau / 6.0, 0, 0.0);
    }
    if (err == OR_OK && nS > 0) err = or_fsi_step(N, c->pos, c->vel, c->mass, S, nS, 0.5 * tau, &fp);
    if (err == OR_OK && nF > 0) err = hhs_level(c, F, nF, 0.5 * tau, level + 1);
    if (err == OR_OK && cross) err = cross_kick(c, S, nS, F, nF, 2.0 * tau / 3.0, 1, tau);
    if (err == OR_OK && nF > 0) err = hhs_level(c, F, nF, 0.5 * tau, level + 1);
    if (err == OR_OK && nS > 0) err = or_fsi_step(N, c->pos, c->vel, c->mass, S, nS, 0.5 * tau, &fp);
    if (err == OR_OK && cross) {
        err = cross_kick(c, S, nS, F, nF, tau / 6.0, 0, 0.0);
        if (err == OR_OK)
            err = pn_kick(N, c->pos, c->vel, c->mass, &fp, S, nS, F, nF, 0, 0.5 * tau);
    }
    free(st); free(S); free(F);
    return err;
}

/* One HHS interval of length tau over all N particles.  level_counts (max_level + 1
 * entries, may be NULL) receives, per level, the number of slow-set particles summed
 * over that level's visits.  Returns OR_ERR_MAXLEVEL (after completing the interval)
 * if some particle wanted a step below the deepest level's pivot. */
int or_hhs_interval(int N, double *pos, double *vel, const double *mass, double tau,
                    const or_hhs_params *p, long long *level_counts)
{
    hhs_ctx c;
    c.N = N; c.pos = pos; c.vel = vel; c.mass = mass; c.p = p;
    c.level_counts = level_counts;
    c.max_level_hit = 0;
    c.step0 = (double *)malloc((size_t)N * sizeof(double));
    int *all = (int *)malloc((size_t)N * sizeof(int));
    if (!c.step0 || !all) { free(c.step0); free(all); return OR_ERR_NOMEM; }
    for (int i = 0; i < N; ++i) all[i] = i;
    if (level_counts) memset(level_counts, 0, (size_t)(p->max_level + 1) * sizeof(long long));
    int err = hhs_level(&c, all, N, tau, 0);
    free(c.step0);
    free(all);
    if (err == OR_OK && c.max_level_hit) err = OR_ERR_MAXLEVEL;
    return err;
}

/* ------------------------------------------------------------------------------- *
 * Adaptive energy-error restarts (Sect. 3.12) around one HHS interval: the state is
 * saved before the interval; if the relative error of the energy E = T + W against its
 * value at the start exceeds eta_restart, the saved state is restored and the interval
 * re-run with every time-step accuracy parameter lowered by 50 % per consecutive restart
 * (eta * 2^-k on attempt k).  An attempt is accepted when its error is within the
 * tolerance, when its error is larger than the previous attempt's ("the energy error
 * starts to increase again": the current result is kept), or after max_restarts
 * restarts.  The caller's parameters stand for the next interval.  *restarts receives the
 * number of restarts, *rel_err the accepted attempt's |Delta E / E|, level_counts its
 * level histogram.  Returns the accepted attempt's status (OR_ERR_MAXLEVEL included).
 * ------------------------------------------------------------------------------- */
int or_hhs_interval_restart(int N, double *pos, double *vel, const double *mass, double tau,
                            const or_hhs_params *p, double eta_restart, int max_restarts,
                            long long *level_counts, int *restarts, double *rel_err)
{
    size_t bytes = 3 * (size_t)N * sizeof(double);
    double *x0 = (double *)malloc(bytes), *v0 = (double *)malloc(bytes);
    if (!x0 || !v0) { free(x0); free(v0); return OR_ERR_NOMEM; }
    memcpy(x0, pos, bytes);
    memcpy(v0, vel, bytes);
    double t0, w0;
    int err = or_energy(N, pos, vel, mass, NULL, N, p->eps2, &t0, &w0);
    double E0 = t0 + w0, prev = INFINITY, e = INFINITY;
    int k = 0;
    for (; err == OR_OK; ++k) {
        or_hhs_params q = *p;
        double f = ldexp(1.0, -k);
        q.eta_ff *= f; q.eta_fb *= f; q.eta_jerk *= f; q.eta_grad *= f; q.eta_va *= f;
        if (k > 0) {
            memcpy(pos, x0, bytes);
            memcpy(vel, v0, bytes);
        }
        int st = or_hhs_interval(N, pos, vel, mass, tau, &q, level_counts);
        if (st != OR_OK && st != OR_ERR_MAXLEVEL) { err = st; break; }
        double t1, w1;
        err = or_energy(N, pos, vel, mass, NULL, N, p->eps2, &t1, &w1);
        if (err != OR_OK) break;
        e = fabs((t1 + w1 - E0) / E0);
        if (e <= eta_restart || (k > 0 && e > prev) || k >= max_restarts) {
            err = st;
            break;
        }
        prev = e;
    }
    *restarts = k;
    *rel_err = e;
    free(x0);
    free(v0);
    return err;
}

/* Time steps of the level-0 set as the interval would assign them (for tests). */
int or_level0_steps(int N, const double *pos, const double *vel, const double *mass,
                    const or_hhs_params *p, double *step)
{
    or_step_params sp = hhs_step_params(p);
    return or_timesteps_all(N, pos, vel, mass, NULL, N, &sp, p->eps2, step);
}

/* =============================================================================== *
 * Adjoint (vector-Jacobian product) of the FSI cycle, hand-derived from the equations
 * of Sect. 2.1.  Notation for a receiver k and a source j != k of the set:
 *   d = r_j - r_k,  s^2 = |d|^2 + eps2,  f(d) = d / s^3,
 *   T(d) = df/dd = I / s^3 - 3 d d^T / s^5             (symmetric, even in d),
 *   Q(d, b) = d(T(d) b)/dd
 *           = -3/s^5 (b d^T + d b^T + (d.b) I) + 15 (d.b) d d^T / s^7   (symmetric).
 * With a_k = sum_j m_j f(d) (Eq. new-newton-acc) and G_k = sum_j m_j T(d)(a_j - a_k)
 * (Eq. new-grad-acc):
 *   VJP of a with cotangent u:
 *     xbar_k = sum_j T(d) (m_k u_j - m_j u_k),   mbar_k = - sum_j u_j . d / s^3
 *   VJP of G through its explicit dependence on r and m (a held fixed), cotangent w:
 *     xbar_k = sum_j Q(d, a_j - a_k) (m_k w_j - m_j w_k),
 *     mbar_k = - sum_j w_j . T(d) (a_j - a_k)
 *   VJP of G through a (cotangent on a):  abar_k = sum_j T(d) (m_k w_j - m_j w_k).
 * =============================================================================== */

/* xbar[:, k] += sx * (VJP of acc)_x,  mbar[k] += sm * (VJP of acc)_m  over the set P,
 * with u a 3 x N array indexed by global id. */
int or_vjp_acc(int N, const double *pos, const double *mass, const int *Pl, int n,
               double eps2, const double *u, double sx, double sm, double *xbar,
               double *mbar)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *UX = u, *UY = u + N, *UZ = u + 2 * (size_t)N;
    int err = OR_OK;
    int q;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (q = 0; q < n; ++q) {
        int k = idx_at(Pl, q);
        double gx = 0, gy = 0, gz = 0, gm = 0;
        for (int l = 0; l < n; ++l) {
            int j = idx_at(Pl, l);
            if (j == k) continue;
            double dx = X[j] - X[k], dy = Y[j] - Y[k], dz = Z[j] - Z[k];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            if (s2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double s = sqrt(s2);
            double is3 = 1.0 / (s2 * s), is5 = is3 / s2;
            double cx = mass[k] * UX[j] - mass[j] * UX[k];
            double cy = mass[k] * UY[j] - mass[j] * UY[k];
            double cz = mass[k] * UZ[j] - mass[j] * UZ[k];
            double dc = dx * cx + dy * cy + dz * cz;
            gx += is3 * cx - 3.0 * is5 * dc * dx;
            gy += is3 * cy - 3.0 * is5 * dc * dy;
            gz += is3 * cz - 3.0 * is5 * dc * dz;
            gm -= (UX[j] * dx + UY[j] * dy + UZ[j] * dz) * is3;
        }
        if (xbar) {
            xbar[k] += sx * gx;
            xbar[(size_t)N + k] += sx * gy;
            xbar[2 * (size_t)N + k] += sx * gz;
        }
        if (mbar) mbar[k] += sm * gm;
    }
    return err;
}

/* xbar, mbar += scale * (VJP of G through r and m, a held fixed), cotangent w, over P.
 * acc: the accelerations inside G (3 x N, global id). */
int or_vjp_grad(int N, const double *pos, const double *mass, const double *acc,
                const int *Pl, int n, double eps2, const double *w, double scale,
                double *xbar, double *mbar)
{
    const double *X = pos, *Y = pos + N, *Z = pos + 2 * (size_t)N;
    const double *AX = acc, *AY = acc + N, *AZ = acc + 2 * (size_t)N;
    const double *WX = w, *WY = w + N, *WZ = w + 2 * (size_t)N;
    int err = OR_OK;
    int q;
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads)
    for (q = 0; q < n; ++q) {
        int k = idx_at(Pl, q);
        double gx = 0, gy = 0, gz = 0, gm = 0;
        for (int l = 0; l < n; ++l) {
            int j = idx_at(Pl, l);
            if (j == k) continue;
            double dx = X[j] - X[k], dy = Y[j] - Y[k], dz = Z[j] - Z[k];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            if (s2 == 0.0) {
#pragma omp atomic write
                err = OR_ERR_COINCIDENT;
                continue;
            }
            double s = sqrt(s2);
            double is3 = 1.0 / (s2 * s), is5 = is3 / s2, is7 = is5 / s2;
            double bx = AX[j] - AX[k], by = AY[j] - AY[k], bz = AZ[j] - AZ[k];
            double cx = mass[k] * WX[j] - mass[j] * WX[k];
            double cy = mass[k] * WY[j] - mass[j] * WY[k];
            double cz = mass[k] * WZ[j] - mass[j] * WZ[k];
            double db = dx * bx + dy * by + dz * bz;
            double dc = dx * cx + dy * cy + dz * cz;
            double bc = bx * cx + by * cy + bz * cz;
            /* Q(d, b) c */
            gx += -3.0 * is5 * (bx * dc + dx * bc + db * cx) + 15.0 * is7 * db * dc * dx;
            gy += -3.0 * is5 * (by * dc + dy * bc + db * cy) + 15.0 * is7 * db * dc * dy;
            gz += -3.0 * is5 * (bz * dc + dz * bc + db * cz) + 15.0 * is7 * db * dc * dz;
            /* -w_j . T(d) b */
            double tbx = is3 * bx - 3.0 * is5 * db * dx;
            double tby = is3 * by - 3.0 * is5 * db * dy;
            double tbz = is3 * bz - 3.0 * is5 * db * dz;
            gm -= WX[j] * tbx + WY[j] * tby + WZ[j] * tbz;
        }
        if (xbar) {
            xbar[k] += scale * gx;
            xbar[(size_t)N + k] += scale * gy;
            xbar[2 * (size_t)N + k] += scale * gz;
        }
        if (mbar) mbar[k] += scale * gm;
    }
    return err;
}

/* Reverse of one or_fsi_step (PN off) of the set P, h, eps2.  Given the input state
 * (pos0, vel0) and the cotangents (gx_out, gv_out) of the output state, writes the
 * cotangents of the input state into gx_in, gv_in (3 x N; entries outside P pass
 * through) and adds the mass cotangent into gm (N).  The forward intermediates are
 * recomputed.  The reverse follows the cycle backwards:
 *   v3 = v2 + h/6 a(x2);  x2 = x1 + h/2 v2;  v2 = v1 + 2h/3 (a(x1) + h^2/24 G(x1));
 *   x1 = x0 + h/2 v1;     v1 = v0 + h/6 a(x0). */
int or_fsi_step_vjp(int N, const double *pos0, const double *vel0, const double *mass,
                    const int *Pl, int n, double h, double eps2,
                    const double *gx_out, const double *gv_out,
                    double *gx_in, double *gv_in, double *gm)
{
    size_t N3 = 3 * (size_t)N;
    double *x1 = (double *)malloc(N3 * sizeof(double));
    double *x2 = (double *)malloc(N3 * sizeof(double));
    double *v1 = (double *)malloc(N3 * sizeof(double));
    double *v2 = (double *)malloc(N3 * sizeof(double));
    double *a0 = (double *)calloc(N3, sizeof(double));
    double *a1 = (double *)calloc(N3, sizeof(double));
    double *g1 = (double *)calloc(N3, sizeof(double));
    double *tmp = (double *)malloc(N3 * sizeof(double));
    double *X = (double *)malloc(N3 * sizeof(double));
    double *V = (double *)malloc(N3 * sizeof(double));
    double *wt = (double *)calloc(N3, sizeof(double));
    double *ab = (double *)calloc(N3, sizeof(double));
    double *u = (double *)calloc(N3, sizeof(double));
    if (!x1 || !x2 || !v1 || !v2 || !a0 || !a1 || !g1 || !tmp || !X || !V || !wt || !ab || !u) {
        free(x1); free(x2); free(v1); free(v2); free(a0); free(a1); free(g1); free(tmp);
        free(X); free(V); free(wt); free(ab); free(u);
        return OR_ERR_NOMEM;
    }
    int err;
    /* forward recompute (global-id arrays) */
    memcpy(x1, pos0, N3 * sizeof(double));
    memcpy(v1, vel0, N3 * sizeof(double));
    err = or_acc(N, pos0, mass, Pl, n, Pl, n, eps2, tmp);
    if (err == OR_OK) {
        scatter3(N, Pl, n, tmp, a0);
        kick(N, v1, Pl, n, tmp, h / 6.0);
        drift(N, x1, v1, Pl, n, 0.5 * h);
        double *gg = (double *)malloc(3 * (size_t)(n > 0 ? n : 1) * sizeof(double));
        if (!gg) err = OR_ERR_NOMEM;
        else {
            err = or_accel_grad(N, x1, mass, Pl, n, Pl, n, eps2, tmp, gg);
            scatter3(N, Pl, n, tmp, a1);
            scatter3(N, Pl, n, gg, g1);
            free(gg);
        }
    }
    if (err == OR_OK) {
        memcpy(v2, v1, N3 * sizeof(double));
        memcpy(x2, x1, N3 * sizeof(double));
        for (int q = 0; q < n; ++q) {
            int k = idx_at(Pl, q);
            for (int c = 0; c < 3; ++c) {
                size_t o = (size_t)c * N + k;
                v2[o] += 2.0 * h / 3.0 * (a1[o] + h * h / 24.0 * g1[o]);
            }
        }
        drift(N, x2, v2, Pl, n, 0.5 * h);
    }
    /* reverse */
    if (err == OR_OK) {
        memcpy(X, gx_out, N3 * sizeof(double));
        memcpy(V, gv_out, N3 * sizeof(double));
        /* v3 = v2 + h/6 a(x2) */
        err = or_vjp_acc(N, x2, mass, Pl, n, eps2, V, h / 6.0, h / 6.0, X, gm);
    }
    if (err == OR_OK) {
        /* x2 = x1 + h/2 v2 */
        for (int q = 0; q < n; ++q) {
            int k = idx_at(Pl, q);
            for (int c = 0; c < 3; ++c) V[(size_t)c * N + k] += 0.5 * h * X[(size_t)c * N + k];
        }
        /* v2 = v1 + 2h/3 a~(x1): cotangent on a~ is wt = 2h/3 V */
        for (int q = 0; q < n; ++q) {
            int k = idx_at(Pl, q);
            for (int c = 0; c < 3; ++c) wt[(size_t)c * N + k] = 2.0 * h / 3.0 * V[(size_t)c * N + k];
        }
        double cg = h * h / 24.0;
        /* abar = cg * (dG/da)^T wt  (same pair form as the acc VJP's position part) */
        err = or_vjp_acc(N, x1, mass, Pl, n, eps2, wt, cg, 0.0, ab, NULL);
        if (err == OR_OK) {
            for (int q = 0; q < n; ++q) {
                int k = idx_at(Pl, q);
                for (int c = 0; c < 3; ++c) {
                    size_t o = (size_t)c * N + k;
                    u[o] = wt[o] + ab[o];
                }
            }
            err = or_vjp_acc(N, x1, mass, Pl, n, eps2, u, 1.0, 1.0, X, gm);
        }
        if (err == OR_OK) err = or_vjp_grad(N, x1, mass, a1, Pl, n, eps2, wt, cg, X, gm);
    }
    if (err == OR_OK) {
        /* x1 = x0 + h/2 v1 */
        for (int q = 0; q < n; ++q) {
            int k = idx_at(Pl, q);
            for (int c = 0; c < 3; ++c) V[(size_t)c * N + k] += 0.5 * h * X[(size_t)c * N + k];
        }
        /* v1 = v0 + h/6 a(x0) */
        err = or_vjp_acc(N, pos0, mass, Pl, n, eps2, V, h / 6.0, h / 6.0, X, gm);
    }
    if (err == OR_OK) {
        memcpy(gx_in, X, N3 * sizeof(double));
        memcpy(gv_in, V, N3 * sizeof(double));
    }
    free(x1); free(x2); free(v1); free(v2); free(a0); free(a1); free(g1); free(tmp);
    free(X); free(V); free(wt); free(ab); free(u);
    return err;
}
