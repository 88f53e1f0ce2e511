/*
 * Plain FP64 CPU oracle for the Tersoff many-body potential.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA path in paper_1710_00882_gb300/.
 *
 * What it computes (Hoehnerbach, Ismail, Bientinesi, "The Tersoff many-body
 * potential: sustainable performance through vectorization", Sec. 2):
 *
 *   E      = 1/2 sum_i sum_{j: r_ij < r_C} f_C(r_ij) [f_R(r_ij) + b_ij f_A(r_ij)]   (Eq. 1, with
 *            Tersoff's 1/2: the paper prints Eq. 1 without it; the 1/2 is what makes diamond Si
 *            come out at the parametrisation's published -4.63 eV/atom)
 *   b_ij   = (1 + beta^n zeta_ij^n)^(-1/(2n))                                       (Eq. 2, eta == n)
 *   zeta_ij= sum_{k != i,j: r_ik < r_C} f_C(r_ik) g(theta_ijk) exp(lambda3 (r_ij - r_ik))   (Eq. 3)
 *
 * and the forces F_m = -dE/dx_m following the loop structure of Algorithm 1 taken
 * literally: for each i, for each neighbour j, a first K loop accumulates zeta_ij,
 * then the pair term V(i,j,zeta_ij) and its r-derivative are applied, then a second K
 * loop re-evaluates each zeta(i,j,k) derivative and scales it by dV/dzeta.
 *
 * The "trivial definitions" the paper omits (Sec. 2) are Tersoff's published forms:
 *   f_C(r) = 1                                  r < R-D
 *          = 1/2 - 1/2 sin(pi (r-R) / (2D))     R-D <= r <= R+D
 *          = 0                                  r > R+D
 *   f_R(r) = A exp(-lambda1 r),   f_A(r) = -B exp(-lambda2 r)
 *   g(theta) = gamma (1 + c^2/d^2 - c^2 / (d^2 + (h - cos theta)^2))
 * The exponent of the lambda3 term is m = 1 as Eq. 3 prints it; a table row with
 * m = 3 selects Tersoff's cubed variant exp((lambda3 (r_ij - r_ik))^3).
 *
 * Parameter table: ntypes^3 rows of 14 doubles, row (ti,tj,tk) at
 * ((ti*nt + tj)*nt + tk), fields {m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D,
 * lambda1, A}.  Two-body terms of the pair (i,j) read row (ti,tj,tj); the three-body term
 * zeta(i,j,k) reads row (ti,tj,tk), including the R, D used for f_C(r_ik).
 *
 * Units: Angstrom, eV, amu, ps.  Orthorhombic periodic box, minimum image.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 14
enum { F_M = 0, F_GAMMA, F_LAM3, F_C, F_D, F_H, F_N, F_BETA, F_LAM2, F_B, F_R, F_DD, F_LAM1, F_A };

static const double PI = 3.14159265358979323846;

static const double *row_of(const double *table, int nt, int a, int b, int c)
{
    return table + ((size_t)((a * nt + b) * nt + c)) * NF;
}

/* d = minimum image of x_j - x_i */
static void min_image(const double *box, const double *xi, const double *xj, double *d)
{
    for (int a = 0; a < 3; ++a) {
        double t = xj[a] - xi[a];
        t -= box[a] * nearbyint(t / box[a]);
        d[a] = t;
    }
}

static double norm3(const double *d) { return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]); }

/* cutoff function f_C and its derivative */
static double f_c(double r, const double *p)
{
    double R = p[F_R], D = p[F_DD];
    if (r < R - D) return 1.0;
    if (r > R + D) return 0.0;
    return 0.5 - 0.5 * sin(PI * (r - R) / (2.0 * D));
}
static double f_c_d(double r, const double *p)
{
    double R = p[F_R], D = p[F_DD];
    if (r < R - D || r > R + D) return 0.0;
    return -0.5 * cos(PI * (r - R) / (2.0 * D)) * PI / (2.0 * D);
}
static double f_r(double r, const double *p) { return p[F_A] * exp(-p[F_LAM1] * r); }
static double f_a(double r, const double *p) { return -p[F_B] * exp(-p[F_LAM2] * r); }

/* angular function g(cos theta) and dg/dcos theta */
static double g_ang(double cost, const double *p)
{
    double c2 = p[F_C] * p[F_C], d2 = p[F_D] * p[F_D], u = p[F_H] - cost;
    return p[F_GAMMA] * (1.0 + c2 / d2 - c2 / (d2 + u * u));
}
static double g_ang_d(double cost, const double *p)
{
    double c2 = p[F_C] * p[F_C], d2 = p[F_D] * p[F_D], u = p[F_H] - cost;
    double den = d2 + u * u;
    return -2.0 * p[F_GAMMA] * c2 * u / (den * den);
}

/* bond order b(zeta) (Eq. 2) and db/dzeta; zeta == 0 gives b = 1, db/dzeta = 0 */
static double b_ij(double zeta, const double *p)
{
    if (zeta <= 0.0) return 1.0;
    double x = pow(p[F_BETA] * zeta, p[F_N]);
    return pow(1.0 + x, -1.0 / (2.0 * p[F_N]));
}
static double b_ij_d(double zeta, const double *p)
{
    if (zeta <= 0.0) return 0.0;
    double x = pow(p[F_BETA] * zeta, p[F_N]);
    double b = pow(1.0 + x, -1.0 / (2.0 * p[F_N]));
    return -0.5 * b / zeta * x / (1.0 + x);
}

/* exponent argument of the lambda3 term and its derivative with respect to (r_ij - r_ik) */
static void lam3_arg(double dr, const double *p, double *arg, double *darg)
{
    double l3 = p[F_LAM3];
    if (p[F_M] == 3.0) {
        double t = l3 * dr;
        *arg = t * t * t;
        *darg = 3.0 * l3 * t * t;
    } else {
        *arg = l3 * dr;
        *darg = l3;
    }
}

/* zeta(i,j,k) of Eq. 3 */
static double zeta_term(const double *dij, double rij, const double *dik, double rik, const double *p)
{
    double cost = (dij[0] * dik[0] + dij[1] * dik[1] + dij[2] * dik[2]) / (rij * rik);
    double arg, darg;
    lam3_arg(rij - rik, p, &arg, &darg);
    return f_c(rik, p) * g_ang(cost, p) * exp(arg);
}

/* derivatives of zeta(i,j,k) with respect to x_i, x_j, x_k */
static void zeta_term_d(const double *dij, double rij, const double *dik, double rik, const double *p,
                        double *dzi, double *dzj, double *dzk)
{
    double uij[3], uik[3];
    for (int a = 0; a < 3; ++a) { uij[a] = dij[a] / rij; uik[a] = dik[a] / rik; }
    double cost = uij[0] * uik[0] + uij[1] * uik[1] + uij[2] * uik[2];
    double arg, darg;
    lam3_arg(rij - rik, p, &arg, &darg);
    double ex = exp(arg);
    double fc = f_c(rik, p), dfc = f_c_d(rik, p);
    double g = g_ang(cost, p), dg = g_ang_d(cost, p);
    for (int a = 0; a < 3; ++a) {
        double dcos_j = (uik[a] - cost * uij[a]) / rij;   /* d cos(theta) / d x_j */
        double dcos_k = (uij[a] - cost * uik[a]) / rik;   /* d cos(theta) / d x_k */
        dzj[a] = fc * ex * (dg * dcos_j + g * darg * uij[a]);
        dzk[a] = dfc * uik[a] * g * ex + fc * ex * (dg * dcos_k - g * darg * uik[a]);
        dzi[a] = -(dzj[a] + dzk[a]);
    }
}

/* pair term V(i,j,zeta) with Tersoff's 1/2, dV/dr_ij at fixed zeta, and dV/dzeta */
static double v_pair(double r, double zeta, const double *p, double *dvdr, double *dvdz)
{
    double fc = f_c(r, p), dfc = f_c_d(r, p);
    double fr = f_r(r, p), fa = f_a(r, p);
    double dfr = -p[F_LAM1] * fr, dfa = -p[F_LAM2] * fa;
    double b = b_ij(zeta, p), db = b_ij_d(zeta, p);
    *dvdr = 0.5 * (dfc * (fr + b * fa) + fc * (dfr + b * dfa));
    *dvdz = 0.5 * fc * fa * db;
    return 0.5 * fc * (fr + b * fa);
}

static double cutoff_of(const double *p) { return p[F_R] + p[F_DD]; }

/*
 * Energy, forces and virial by Algorithm 1.
 *   pos[N][3], types[N] in [0,ntypes), box[3]; neighbour list in CSR form (offsets[N+1],
 *   idx[offsets[N]]) holding, for each i, every j != i within some radius >= max r_C.
 *   Outputs: *energy (eV), forces[N][3] (eV/A, overwritten), virial[9] (row-major
 *   W_ab = sum over terms of d_a F_b with d relative to i; may be NULL).
 * Returns 0, or -1 on a bad argument.
 */
int oracle_energy_forces(int64_t N, const double *pos, const int32_t *types, const double *box, int ntypes,
                         const double *table, const int64_t *offsets, const int32_t *idx, double *energy,
                         double *forces, double *virial)
{
    if (N < 0 || ntypes < 1) return -1;
    double E = 0.0, W[9] = {0};
    memset(forces, 0, sizeof(double) * 3 * (size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        const double *xi = pos + 3 * i;
        int ti = types[i];
        for (int64_t jj = offsets[i]; jj < offsets[i + 1]; ++jj) {
            int64_t j = idx[jj];
            int tj = types[j];
            const double *pij = row_of(table, ntypes, ti, tj, tj);
            double dij[3];
            min_image(box, xi, pos + 3 * j, dij);
            double rij = norm3(dij);
            if (rij >= cutoff_of(pij)) continue;

            /* first K loop: zeta_ij */
            double zeta = 0.0;
            for (int64_t kk = offsets[i]; kk < offsets[i + 1]; ++kk) {
                int64_t k = idx[kk];
                if (k == j) continue;
                const double *pijk = row_of(table, ntypes, ti, tj, types[k]);
                double dik[3];
                min_image(box, xi, pos + 3 * k, dik);
                double rik = norm3(dik);
                if (rik >= cutoff_of(pijk)) continue;
                zeta += zeta_term(dij, rij, dik, rik, pijk);
            }

            /* pair term */
            double dvdr, dvdz;
            E += v_pair(rij, zeta, pij, &dvdr, &dvdz);
            for (int a = 0; a < 3; ++a) {
                double fj = -dvdr * dij[a] / rij; /* -dV/dx_j */
                forces[3 * j + a] += fj;
                forces[3 * i + a] -= fj;          /* -dV/dx_i = +dV/dx_j */
            }
            if (virial)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) W[3 * a + b] += dij[a] * (-dvdr * dij[b] / rij);

            /* second K loop: zeta derivatives scaled by dV/dzeta */
            for (int64_t kk = offsets[i]; kk < offsets[i + 1]; ++kk) {
                int64_t k = idx[kk];
                if (k == j) continue;
                const double *pijk = row_of(table, ntypes, ti, tj, types[k]);
                double dik[3];
                min_image(box, xi, pos + 3 * k, dik);
                double rik = norm3(dik);
                if (rik >= cutoff_of(pijk)) continue;
                double dzi[3], dzj[3], dzk[3];
                zeta_term_d(dij, rij, dik, rik, pijk, dzi, dzj, dzk);
                for (int a = 0; a < 3; ++a) {
                    forces[3 * i + a] -= dvdz * dzi[a];
                    forces[3 * j + a] -= dvdz * dzj[a];
                    forces[3 * k + a] -= dvdz * dzk[a];
                }
                if (virial)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            W[3 * a + b] += dij[a] * (-dvdz * dzj[b]) + dik[a] * (-dvdz * dzk[b]);
            }
        }
    }
    *energy = E;
    if (virial) memcpy(virial, W, sizeof W);
    return 0;
}

/*
 * Brute-force O(N^2) neighbour search: for each i, every j != i with minimum-image
 * distance < rcut, in ascending j.  offsets[N+1] is always written; idx is written up to
 * cap entries.  Returns the total number of entries (callers retry with a larger cap when
 * the return exceeds cap), or -1 on a bad argument.
 */
int64_t oracle_neighbors_brute(int64_t N, const double *pos, const double *box, double rcut, int64_t *offsets,
                               int32_t *idx, int64_t cap)
{
    if (N < 0 || rcut <= 0) return -1;
    int64_t n = 0;
    double rc2 = rcut * rcut;
    for (int64_t i = 0; i < N; ++i) {
        offsets[i] = n;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(box, pos + 3 * i, pos + 3 * j, d);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) {
                if (n < cap) idx[n] = (int32_t)j;
                ++n;
            }
        }
    }
    offsets[N] = n;
    return n;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Linked-cell neighbour search with the same output as oracle_neighbors_brute (each list
 * sorted ascending).  Needs at least 3 cells of edge >= rcut per dimension; returns -2 when
 * the box is too small for that (use the brute-force search instead).
 */
int64_t oracle_neighbors_cells(int64_t N, const double *pos, const double *box, double rcut, int64_t *offsets,
                               int32_t *idx, int64_t cap)
{
    if (N < 0 || rcut <= 0) return -1;
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(box[a] / rcut);
        if (nc[a] < 3) return -2;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int *cell_of = malloc(sizeof(int) * 3 * (size_t)(N > 0 ? N : 1));
    int32_t *tmp = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!head || !next || !cell_of || !tmp) {
        free(head); free(next); free(cell_of); free(tmp);
        return -1;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = N - 1; i >= 0; --i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            double s = pos[3 * i + a] / box[a];
            s -= floor(s);
            int q = (int)(s * nc[a]);
            if (q >= nc[a]) q = nc[a] - 1;
            if (q < 0) q = 0;
            ci[a] = q;
            cell_of[3 * i + a] = q;
        }
        int64_t c = ((int64_t)ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
        next[i] = head[c];
        head[c] = i;
    }
    double rc2 = rcut * rcut;
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) {
        offsets[i] = n;
        int64_t m = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = (cell_of[3 * i] + dx + nc[0]) % nc[0];
                    int cy = (cell_of[3 * i + 1] + dy + nc[1]) % nc[1];
                    int cz = (cell_of[3 * i + 2] + dz + nc[2]) % nc[2];
                    int64_t c = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                    for (int64_t j = head[c]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double d[3];
                        min_image(box, pos + 3 * i, pos + 3 * j, d);
                        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) tmp[m++] = (int32_t)j;
                    }
                }
        qsort(tmp, (size_t)m, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < m; ++q) {
            if (n + q < cap) idx[n + q] = tmp[q];
        }
        n += m;
    }
    offsets[N] = n;
    free(head); free(next); free(cell_of); free(tmp);
    return n;
}

/* largest r_C = R + D over the table */
static double max_cutoff(int ntypes, const double *table)
{
    double rc = 0.0;
    for (int r = 0; r < ntypes * ntypes * ntypes; ++r) {
        double c = table[(size_t)r * NF + F_R] + table[(size_t)r * NF + F_DD];
        if (c > rc) rc = c;
    }
    return rc;
}

/* neighbour list at exactly the largest cutoff, by cells when the box allows, else brute force */
static int64_t build_list(int64_t N, const double *pos, const double *box, double rc, int64_t *offsets,
                          int32_t **idx, int64_t *cap)
{
    for (;;) {
        int64_t n = oracle_neighbors_cells(N, pos, box, rc, offsets, *idx, *cap);
        if (n == -2) n = oracle_neighbors_brute(N, pos, box, rc, offsets, *idx, *cap);
        if (n < 0) return n;
        if (n <= *cap) return n;
        free(*idx);
        *cap = n + n / 4 + 16;
        *idx = malloc(sizeof(int32_t) * (size_t)*cap);
        if (!*idx) return -1;
    }
}

/* eV/(A*amu) -> A/ps^2, from the SI values of the electronvolt and the atomic mass unit:
 * (J / 1e-10 m) / kg = m/s^2, and 1 m/s^2 = 1e10 A / 1e24 ps^2, so the factor is 1e-4. */
static const double EV_J = 1.602176634e-19;
static const double AMU_KG = 1.66053906660e-27;
static double accel_unit(void) { return EV_J / AMU_KG * 1e-4; }

/* kinetic energy in eV: sum 1/2 m v^2 with v in A/ps and m in amu */
double oracle_kinetic(int64_t N, const double *vel, const int32_t *types, const double *masses)
{
    double ke = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double m = masses[types[i]];
        const double *v = vel + 3 * i;
        ke += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
    return ke / accel_unit();
}

/*
 * Velocity-Verlet NVE: v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m, nsteps times.
 * The neighbour list is rebuilt every step at exactly the largest cutoff, so no skin is
 * involved.  pos and vel are updated in place (positions are not wrapped).  trace, when
 * not NULL, receives [nsteps+1][2] = (potential, kinetic) energy after each step
 * (row 0 = initial state).  Returns 0 or a negative error.
 */
int oracle_md_run(int64_t N, double *pos, double *vel, const int32_t *types, const double *box, int ntypes,
                  const double *table, const double *masses, double dt, int64_t nsteps, double *trace)
{
    if (N <= 0 || nsteps < 0) return -1;
    double rc = max_cutoff(ntypes, table);
    int64_t cap = 32 * N;
    int64_t *offsets = malloc(sizeof(int64_t) * (size_t)(N + 1));
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)cap);
    double *F = malloc(sizeof(double) * 3 * (size_t)N);
    if (!offsets || !idx || !F) {
        free(offsets); free(idx); free(F);
        return -1;
    }
    const double acc = accel_unit();
    double E;
    int rc_err = 0;
    if (build_list(N, pos, box, rc, offsets, &idx, &cap) < 0) { rc_err = -1; goto done; }
    oracle_energy_forces(N, pos, types, box, ntypes, table, offsets, idx, &E, F, NULL);
    if (trace) { trace[0] = E; trace[1] = oracle_kinetic(N, vel, types, masses); }
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < N; ++i) {
            double c = 0.5 * dt * acc / masses[types[i]];
            for (int a = 0; a < 3; ++a) {
                vel[3 * i + a] += c * F[3 * i + a];
                pos[3 * i + a] += dt * vel[3 * i + a];
            }
        }
        if (build_list(N, pos, box, rc, offsets, &idx, &cap) < 0) { rc_err = -1; goto done; }
        oracle_energy_forces(N, pos, types, box, ntypes, table, offsets, idx, &E, F, NULL);
        for (int64_t i = 0; i < N; ++i) {
            double c = 0.5 * dt * acc / masses[types[i]];
            for (int a = 0; a < 3; ++a) vel[3 * i + a] += c * F[3 * i + a];
        }
        if (trace) { trace[2 * s] = E; trace[2 * s + 1] = oracle_kinetic(N, vel, types, masses); }
    }
done:
    free(offsets); free(idx); free(F);
    return rc_err;
}

/* the acceleration unit used above, exported so tests can pin it against its definition */
double oracle_accel_unit(void) { return accel_unit(); }
