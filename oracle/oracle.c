/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the GENGA long-range kick path.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load this file's library.  It
 * shares no source, header, table or helper with the CUDA path.
 *
 * Paper: Brasser, Grimm, Hatalova & Stadel (2023), "Speeding up the GENGA
 * N-body integrator on consumer-grade graphics cards".  What it computes:
 *
 *   critical radius       Sect. 1, Eq. (1):  r_crit,i = max(n1 R_H,i, n2 dt v_i),
 *                         R_H,i = a_i (m_i / 3 M*)^(1/3)
 *   changeover weight K   Sect. 1 (the smooth switch of the hybrid
 *                         symplectic integrator; Chambers 1999 form)
 *   long-range kick       Sect. 1 (the N^2 force terms):
 *                         a_i = sum_{j!=i} G m_j K (x_j - x_i) / |x_j - x_i|^3
 *   encounter pairs       Sect. 1 (pairs inside the changeover radius)
 *   Kepler drift          Sect. 1 (always FP64): universal-variable f and g
 *   close-encounter level Sect. 1 (level 1 of the hybrid integrator): the
 *                         connected groups of encounter pairs are integrated
 *                         over the drift with a Bulirsch-Stoer method under the
 *                         central body and the (1 - K) part of their mutual forces
 *   intermediate levels   Sect. 1 (the multi-level changeover): symplectic
 *                         sub-steps between the kick and the Bulirsch-Stoer
 *                         level, each level with its own changeover radius
 *   mergers, removal      Sect. 2: collisions are perfect mergers; bodies closer
 *                         than r_in to or farther than r_out from the central
 *                         body are removed (both leave a massless "ghost")
 *   energy / ang. mom.    Sect. 3.1: dE/E = E(t)/E0 - 1, dL/L = L(t)/L0 - 1
 *
 * Readings where the paper is silent: democratic-heliocentric coordinates (heliocentric x, barycentric
 * v; Kepler mu = G M*; the central-body momentum drift x += tau P / M*);
 * the Kepler velocity of Eq. (1) is the heliocentric speed v + P/M*;
 * a_i is the osculating semi-major axis with mu_i = G (M* + m_i), and
 * r_i replaces a_i for unbound orbits; the pair radius is
 * max(r_crit,i, r_crit,j) (mode 0) or n1 ((m_i+m_j)/3M*)^(1/3) (a_i+a_j)/2,
 * three mutual Hill radii (mode 1); y = (r/r_crit,ij - 0.1)/0.9 with
 * K(y) = y^2/(2y^2 - 2y + 1) (form 0) or 10y^3 - 15y^4 + 6y^5 (form 1),
 * K = 0 for y <= 0 and 1 for y >= 1; an encounter is r_ij < r_crit,ij.
 *
 * Every sum over all bodies is Neumaier-compensated in index order, so the
 * result does not depend on the number of OpenMP threads; the group forces
 * of the close-encounter level are plain sums in index order (a group holds
 * a few bodies).
 * Build: cc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- sums -- */

typedef struct { double s, c; } nsum;   /* Neumaier (1974) running sum */

static void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                       a->c += (v - t) + a->s;
    a->s = t;
}

static double nval(const nsum *a) { return a->s + a->c; }

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------- changeover (Sect. 1) */

/* K(y): 0 for y <= 0, 1 for y >= 1, smooth in between. */
double oracle_changeover(double y, int form)
{
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    if (form == 0) {
        double y2 = y * y;
        return y2 / (2.0 * y2 - 2.0 * y + 1.0);
    }
    return y * y * y * (10.0 - 15.0 * y + 6.0 * y * y);
}

/* ------------------------------------------------ total momentum P -------- */

/* P = sum_j m_j v_j (barycentric momenta of the non-central bodies). */
void oracle_momentum(int N, const double *vx, const double *vy, const double *vz,
                     const double *m, double *P)
{
    nsum px = {0, 0}, py = {0, 0}, pz = {0, 0};
    for (int j = 0; j < N; j++) {
        nadd(&px, m[j] * vx[j]);
        nadd(&py, m[j] * vy[j]);
        nadd(&pz, m[j] * vz[j]);
    }
    P[0] = nval(&px); P[1] = nval(&py); P[2] = nval(&pz);
}

/* ------------------------------------------- critical radius, Eq. (1) ----- */

/*
 * Per body: the osculating semi-major axis a_i (1/a = 2/r - v_hel^2/mu_i,
 * mu_i = G (M* + m_i); a_i = r_i when 1/a <= 0) and the Eq. (1) radius
 * r_crit,i = max(n1 a_i (m_i/3M*)^(1/3), n2 dt |v_hel,i|), v_hel = v + P/M*.
 */
void oracle_rcrit(int N, const double *x, const double *y, const double *z,
                  const double *vx, const double *vy, const double *vz, const double *m,
                  double G, double Mstar, double dt, double n1, double n2,
                  double *a_out, double *rc_out)
{
    double P[3];
    oracle_momentum(N, vx, vy, vz, m, P);
    for (int i = 0; i < N; i++) {
        double ux = vx[i] + P[0] / Mstar;
        double uy = vy[i] + P[1] / Mstar;
        double uz = vz[i] + P[2] / Mstar;
        double v2 = ux * ux + uy * uy + uz * uz;
        double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
        double mu = G * (Mstar + m[i]);
        double inva = 2.0 / r - v2 / mu;
        double a = (inva > 0.0) ? 1.0 / inva : r;
        double RH = a * cbrt(m[i] / (3.0 * Mstar));
        double t1 = n1 * RH, t2 = n2 * dt * sqrt(v2);
        a_out[i] = a;
        rc_out[i] = (t1 > t2) ? t1 : t2;
    }
}

/* Pair radius: mode 0 = max of the Eq. (1) radii; mode 1 = n1 mutual Hill radii. */
double oracle_pair_rcrit(int mode, double mi, double mj, double ai, double aj,
                         double rci, double rcj, double n1, double Mstar)
{
    if (mode == 0) return (rci > rcj) ? rci : rcj;
    return n1 * cbrt((mi + mj) / (3.0 * Mstar)) * 0.5 * (ai + aj);
}

/* ---------------------------------------------- long-range kick (Sect. 1) -- */

/*
 * Test-particle mode 2 (Sect. 3, the giant-planet runs): with n_big >= 0,
 * bodies n_big..N-1 are test particles that feel the bodies 0..n_big-1 but
 * not each other, while those feel everything; a pair of two test particles
 * has no force, no encounter and no potential energy.  n_big < 0: every pair
 * interacts.
 */
static int tp_pair(int n_big, int i, int j)
{
    return n_big >= 0 && i >= n_big && j >= n_big;
}

/*
 * Accelerations of the bodies listed in idx[0..nidx): the direct sum over
 * all j != i of G m_j K(y_ij) (x_j - x_i)/r_ij^3.  Optional absout[k] gets
 * sum_j |a_ij| (the conditioning of body idx[k]'s sum).
 */
void oracle_kick_acc(int N, const double *x, const double *y, const double *z,
                     const double *m, const double *a, const double *rc,
                     double G, double Mstar, double n1, int mode, int form, int n_big,
                     int nidx, const int64_t *idx,
                     double *ax, double *ay, double *az, double *absout)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < nidx; k++) {
        int i = (int)idx[k];
        nsum sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sa = {0, 0};
        for (int j = 0; j < N; j++) {
            if (j == i || tp_pair(n_big, i, j)) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;          /* coincident bodies: no direction, no force */
            double r = sqrt(r2);
            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);
            double K = 1.0;
            if (r < rcij) K = oracle_changeover((r / rcij - 0.1) / 0.9, form);
            if (K == 0.0) continue;
            double f = G * m[j] * K / (r2 * r);
            nadd(&sx, f * dx);
            nadd(&sy, f * dy);
            nadd(&sz, f * dz);
            nadd(&sa, fabs(f) * r);
        }
        ax[k] = nval(&sx); ay[k] = nval(&sy); az[k] = nval(&sz);
        if (absout) absout[k] = nval(&sa);
    }
}

/* Kick: r_crit from the current state, then v_i += a_i tau for all i. */
void oracle_kick(int N, const double *x, const double *y, const double *z,
                 double *vx, double *vy, double *vz, const double *m,
                 double G, double Mstar, double dt, double n1, double n2, int mode, int form,
                 int n_big, double tau, double *ax, double *ay, double *az)
{
    double *a = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    double *rc = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    oracle_rcrit(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, a, rc);
    for (int i = 0; i < N; i++) idx[i] = i;
    oracle_kick_acc(N, x, y, z, m, a, rc, G, Mstar, n1, mode, form, n_big, N, idx, ax, ay, az, NULL);
    for (int i = 0; i < N; i++) {
        vx[i] += ax[i] * tau;
        vy[i] += ay[i] * tau;
        vz[i] += az[i] * tau;
    }
    free(a); free(rc); free(idx);
}

/* ------------------------------------------- encounter pairs (Sect. 1) ---- */

/*
 * All pairs i < j with r_ij < r_crit,ij, in lexicographic order.  Writes at
 * most `cap` pairs to pairs[2k], pairs[2k+1]; returns the true count.  Pairs
 * with |r_ij - r_crit,ij| <= band * r_crit,ij (either side) also go to
 * band_pairs (at most band_cap; true count in *band_count).
 */
int64_t oracle_encounters(int N, const double *x, const double *y, const double *z,
                          const double *m, const double *a, const double *rc,
                          double n1, double Mstar, int mode, int n_big,
                          int32_t *pairs, int64_t cap, double band,
                          int32_t *band_pairs, int64_t band_cap, int64_t *band_count)
{
    int64_t cnt = 0, bcnt = 0;
    for (int i = 0; i < N; i++) {
        for (int j = i + 1; j < N; j++) {
            if (tp_pair(n_big, i, j)) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);
            if (r < rcij) {
                if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                cnt++;
            }
            if (fabs(r - rcij) <= band * rcij) {
                if (bcnt < band_cap) { band_pairs[2 * bcnt] = i; band_pairs[2 * bcnt + 1] = j; }
                bcnt++;
            }
        }
    }
    if (band_count) *band_count = bcnt;
    return cnt;
}

/*
 * Predicted entries (reading of the close-encounter level's grouping): a pair
 * not inside r_crit,ij yet (r_ij >= r_crit,ij) but within PREDICT_RANGE
 * r_crit,ij whose straight-line relative motion over the coming drift,
 * d + u t with d = x_j - x_i, u = v_j - v_i (the state the list is built
 * from) and t between 0 and dt, comes closer than r_crit,ij.  Such pairs join
 * the groups of that drift (they are not encounter pairs).  Writes at most
 * `cap` pairs (i < j, lexicographic); returns the true count.
 */
#define PREDICT_RANGE 1.5

int64_t oracle_predicted_pairs(int N, const double *x, const double *y, const double *z,
                               const double *vx, const double *vy, const double *vz,
                               const double *m, const double *a, const double *rc,
                               double n1, double Mstar, int mode, int n_big, double dt,
                               int32_t *pairs, int64_t cap)
{
    int64_t cnt = 0;
    double tlo = dt < 0.0 ? dt : 0.0, thi = dt < 0.0 ? 0.0 : dt;
    for (int i = 0; i < N; i++) {
        for (int j = i + 1; j < N; j++) {
            if (tp_pair(n_big, i, j)) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);
            if (r < rcij || r >= PREDICT_RANGE * rcij) continue;
            double ux = vx[j] - vx[i], uy = vy[j] - vy[i], uz = vz[j] - vz[i];
            double uu = ux * ux + uy * uy + uz * uz, du = dx * ux + dy * uy + dz * uz;
            double t = uu > 0.0 ? -du / uu : 0.0;
            if (t < tlo) t = tlo;
            if (t > thi) t = thi;
            double px = dx + ux * t, py = dy + uy * t, pz = dz + uz * t;
            if (px * px + py * py + pz * pz < rcij * rcij) {
                if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                cnt++;
            }
        }
    }
    return cnt;
}

/* ------------------------------------------- Kepler drift (Sect. 1) ------- */

/*
 * Stumpff functions c0..c3 of z by Danby's method (Fundamentals of
 * Celestial Mechanics, 2nd ed., Sect. 6.9): reduce z by powers of four
 * until |z| <= 0.1, sum the series of c2 and c3, then undo the reduction
 * with the quadruple-argument relations.
 */
static void stumpff(double z, double *c0, double *c1, double *c2, double *c3)
{
    int n = 0;
    while (fabs(z) > 0.1) { z *= 0.25; n++; }
    double s3 = (1.0 - z / 20.0 * (1.0 - z / 42.0 * (1.0 - z / 72.0 * (1.0 - z / 110.0 *
                (1.0 - z / 156.0 * (1.0 - z / 210.0)))))) / 6.0;
    double s2 = (1.0 - z / 12.0 * (1.0 - z / 30.0 * (1.0 - z / 56.0 * (1.0 - z / 90.0 *
                (1.0 - z / 132.0 * (1.0 - z / 182.0)))))) / 2.0;
    double s1 = 1.0 - z * s3;
    double s0 = 1.0 - z * s2;
    for (; n > 0; n--) {
        s3 = (s2 + s0 * s3) * 0.25;
        s2 = s1 * s1 * 0.5;
        s1 = s1 * s0;
        s0 = 2.0 * s0 * s0 - 1.0;
    }
    *c0 = s0; *c1 = s1; *c2 = s2; *c3 = s3;
}

/*
 * Two-body drift of one body about mu for time dt, universal variables.
 * Kepler's equation in the universal anomaly s,
 *   F(s) = r0 G1 + eta0 G2 + mu G3 - dt = 0,   G_k = s^k c_k(beta s^2),
 * beta = 2 mu / r0 - v0^2, eta0 = x0.v0, is solved by the Laguerre-Conway
 * iteration (n = 5) from s = dt / r0; then the f and g functions give
 *   x = f x0 + g v0,  v = fdot x0 + gdot v0.
 * The iteration converges cubically, so a step |ds| <= 1e-12 |s| leaves the
 * new iterate at rounding level.  Returns 0 when that happens within
 * max_iter steps, else 1 (the state is still advanced with the last iterate).
 */
int oracle_kepler(double mu, double *xv, double dt, int max_iter)
{
    double x0 = xv[0], y0 = xv[1], z0 = xv[2], u0 = xv[3], v0 = xv[4], w0 = xv[5];
    double r0 = sqrt(x0 * x0 + y0 * y0 + z0 * z0);
    double vv = u0 * u0 + v0 * v0 + w0 * w0;
    double eta = x0 * u0 + y0 * v0 + z0 * w0;
    double beta = 2.0 * mu / r0 - vv;
    double s = dt / r0;
    double c0, c1, c2, c3;
    int status = 1;
    for (int it = 0; it < max_iter; it++) {
        stumpff(beta * s * s, &c0, &c1, &c2, &c3);
        double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
        double F = r0 * G1 + eta * G2 + mu * G3 - dt;
        double Fp = r0 * c0 + eta * G1 + mu * G2;
        double Fpp = eta * c0 + (mu - beta * r0) * G1;
        double disc = 16.0 * Fp * Fp - 20.0 * F * Fpp;
        double den = Fp + copysign(sqrt(fabs(disc)), Fp);
        double ds = -5.0 * F / den;
        s += ds;
        if (fabs(ds) <= 1e-12 * fabs(s)) { status = 0; break; }
    }
    stumpff(beta * s * s, &c0, &c1, &c2, &c3);
    double G1 = s * c1, G2 = s * s * c2;
    double r = r0 * c0 + eta * G1 + mu * G2;
    double f = 1.0 - mu * G2 / r0;
    double g = r0 * G1 + eta * G2;
    double fd = -mu * G1 / (r * r0);
    double gd = 1.0 - mu * G2 / r;
    xv[0] = f * x0 + g * u0;  xv[1] = f * y0 + g * v0;  xv[2] = f * z0 + g * w0;
    xv[3] = fd * x0 + gd * u0; xv[4] = fd * y0 + gd * v0; xv[5] = fd * z0 + gd * w0;
    return status;
}

/* Central-body momentum drift: x_i += tau P / M*, P = sum_j m_j v_j. */
void oracle_hc_drift(int N, double *x, double *y, double *z,
                     const double *vx, const double *vy, const double *vz, const double *m,
                     double Mstar, double tau)
{
    double P[3];
    oracle_momentum(N, vx, vy, vz, m, P);
    for (int i = 0; i < N; i++) {
        x[i] += tau * P[0] / Mstar;
        y[i] += tau * P[1] / Mstar;
        z[i] += tau * P[2] / Mstar;
    }
}

/* Drift of the step: HC(dt/2), Kepler(dt) with mu = G M*, HC(dt/2).
 * Returns the number of bodies whose Kepler solve did not converge. */
int oracle_drift(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                 const double *m, double G, double Mstar, double dt, int max_iter)
{
    int bad = 0;
    oracle_hc_drift(N, x, y, z, vx, vy, vz, m, Mstar, 0.5 * dt);
    #pragma omp parallel for reduction(+:bad)
    for (int i = 0; i < N; i++) {
        double s[6] = {x[i], y[i], z[i], vx[i], vy[i], vz[i]};
        bad += oracle_kepler(G * Mstar, s, dt, max_iter);
        x[i] = s[0]; y[i] = s[1]; z[i] = s[2];
        vx[i] = s[3]; vy[i] = s[4]; vz[i] = s[5];
    }
    oracle_hc_drift(N, x, y, z, vx, vy, vz, m, Mstar, 0.5 * dt);
    return bad;
}

/* Level-0 step, kick(dt/2) drift(dt) kick(dt/2), repeated nsteps times.
 * Returns the total count of non-converged Kepler solves. */
int oracle_step(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                const double *m, double G, double Mstar, double dt, double n1, double n2,
                int mode, int form, int n_big, int max_iter, int nsteps)
{
    int bad = 0;
    size_t n = (size_t)(N > 0 ? N : 1);
    double *ax = (double *)malloc(sizeof(double) * n);
    double *ay = (double *)malloc(sizeof(double) * n);
    double *az = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; s++) {
        oracle_kick(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, mode, form, n_big, 0.5 * dt, ax, ay, az);
        bad += oracle_drift(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, max_iter);
        oracle_kick(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, mode, form, n_big, 0.5 * dt, ax, ay, az);
    }
    free(ax); free(ay); free(az);
    return bad;
}

/* --------------------------------- close-encounter level (Sect. 1) ------- */

/*
 * Groups: the connected components of the graph whose edges are the
 * encounter pairs.  label[v] = the smallest body index in v's component for
 * every body that appears in a pair, -1 for every other body.  Plain
 * union-find (each union hangs the larger root under the smaller one).
 * Returns the number of groups.
 */
static int uf_root(int32_t *parent, int v)
{
    while (parent[v] != v) v = parent[v];
    return v;
}

int oracle_groups(int N, int64_t npairs, const int32_t *pairs, int32_t *label)
{
    for (int v = 0; v < N; v++) label[v] = -1;
    for (int64_t p = 0; p < npairs; p++) {
        label[pairs[2 * p]] = pairs[2 * p];
        label[pairs[2 * p + 1]] = pairs[2 * p + 1];
    }
    for (int64_t p = 0; p < npairs; p++) {
        int ri = uf_root(label, pairs[2 * p]), rj = uf_root(label, pairs[2 * p + 1]);
        if (ri < rj) label[rj] = ri;
        else if (rj < ri) label[ri] = rj;
    }
    int ngroups = 0;
    for (int v = 0; v < N; v++) {
        if (label[v] < 0) continue;
        label[v] = uf_root(label, v);   /* roots are smaller than v: already final */
        if (label[v] == v) ngroups++;
    }
    return ngroups;
}

/*
 * Levels of the changeover (Sect. 1: intermediate levels between the
 * symplectic step and the Bulirsch-Stoer integrator, each a symplectic step
 * with a smaller time step).  Readings: with L intermediate levels and s
 * sub-steps per level, level l (0 <= l <= L) has the time step dt / s^l and
 * the pair radius r_crit,l = r_crit,ij / s^l (the velocity term of Eq. 1
 * shrinks with the step); K_l(r) = K((r / r_crit,l - 0.1) / 0.9).  The pair
 * force is split into
 *   level l <= L:           W_l = K_l prod_{k<l} (1 - K_k)
 *   Bulirsch-Stoer (L + 1): W_{L+1} = prod_{k<=L} (1 - K_k),
 * which add up to 1 (the products telescope); W_0 = K_0 is the kick's
 * weight.  s^l is an exact integer, so r_crit,l is one rounded quotient.
 */
double oracle_ml_radius(double rc, int l, int s)
{
    double p = 1.0;
    for (int k = 0; k < l; k++) p *= s;
    return rc / p;
}

double oracle_ml_weight(double q, double rc, int l, int L, int s, int form)
{
    double w = 1.0;
    for (int k = 0; k < l && k <= L; k++)
        w *= 1.0 - oracle_changeover((q / oracle_ml_radius(rc, k, s) - 0.1) / 0.9, form);
    if (l <= L) w *= oracle_changeover((q / oracle_ml_radius(rc, l, s) - 0.1) / 0.9, form);
    return w;
}

/*
 * One group of n bodies (body indices mem[0] < mem[1] < ...).  What the
 * Bulirsch-Stoer level integrates over the drift (the level-1 Hamiltonian
 * of the hybrid step): every member moves about the central body
 * (mu = G M*, as in the Kepler drift) and feels the other members through
 * the part of their pair force the kick leaves out,
 *   dv_i/dt = -mu x_i/|x_i|^3 + sum_{j in group} G m_j (1 - K(y_ij)) (x_j - x_i)/r_ij^3,
 * with r_crit,ij from the a_i, r_crit,i of the step's first kick (fixed over
 * the drift), so that kick + group force = the whole Newtonian pair force.
 */
typedef struct {
    int n;
    const int32_t *mem;
    const double *m, *a, *rc;
    double G, Mstar, n1;
    int mode, form, n_big;
    const int32_t *ghost;   /* per member: merged away (no force either way); NULL: none */
    int nlev, nsub;         /* intermediate levels L and sub-steps s (0, 1: none) */
} bs_group;

static int bs_ghost(const bs_group *g, int k) { return g->ghost && g->ghost[k]; }

/* State layout: s[6k + 0..2] = position, s[6k + 3..5] = velocity of member k. */
static void bs_deriv(const bs_group *g, const double *s, double *ds)
{
    for (int i = 0; i < g->n; i++) {
        const double *xi = s + 6 * i;
        int bi = g->mem[i];
        double r2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        double r = sqrt(r2);
        double c = -g->G * g->Mstar / (r2 * r);
        double ax = c * xi[0], ay = c * xi[1], az = c * xi[2];
        for (int j = 0; j < g->n; j++) {
            int bj = g->mem[j];
            if (j == i || tp_pair(g->n_big, bi, bj) || bs_ghost(g, i) || bs_ghost(g, j)) continue;
            const double *xj = s + 6 * j;
            double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
            double q2 = dx * dx + dy * dy + dz * dz;
            if (q2 == 0.0) continue;
            double q = sqrt(q2);
            double rcij = oracle_pair_rcrit(g->mode, g->m[bi], g->m[bj], g->a[bi], g->a[bj],
                                            g->rc[bi], g->rc[bj], g->n1, g->Mstar);
            if (q >= oracle_ml_radius(rcij, g->nlev, g->nsub)) continue;   /* the kicks have all of it */
            double w = oracle_ml_weight(q, rcij, g->nlev + 1, g->nlev, g->nsub, g->form);
            double f = g->G * g->m[bj] * w / (q2 * q);
            ax += f * dx;
            ay += f * dy;
            az += f * dz;
        }
        double *d = ds + 6 * i;
        d[0] = xi[3]; d[1] = xi[4]; d[2] = xi[5];
        d[3] = ax;    d[4] = ay;    d[5] = az;
    }
}

/* The level-1 acceleration of each member of a group (bs_deriv's velocity
 * half) at the given state: acc[3k + c] for member k; below nlev intermediate
 * levels of nsub sub-steps (0, 1: none). */
void oracle_bs_acc_ml(int n, const int32_t *mem, const double *x, const double *y, const double *z,
                      const double *m, const double *a, const double *rc, double G, double Mstar,
                      double n1, int mode, int form, int n_big, int nlev, int nsub, double *acc)
{
    bs_group g = {n, mem, m, a, rc, G, Mstar, n1, mode, form, n_big, NULL, nlev, nsub};
    double *s = (double *)calloc((size_t)(6 * n > 0 ? 6 * n : 1), sizeof(double));
    double *ds = (double *)calloc((size_t)(6 * n > 0 ? 6 * n : 1), sizeof(double));
    for (int k = 0; k < n; k++) {
        s[6 * k] = x[mem[k]]; s[6 * k + 1] = y[mem[k]]; s[6 * k + 2] = z[mem[k]];
    }
    bs_deriv(&g, s, ds);
    for (int k = 0; k < n; k++)
        for (int c = 0; c < 3; c++) acc[3 * k + c] = ds[6 * k + 3 + c];
    free(s);
    free(ds);
}

void oracle_bs_acc(int n, const int32_t *mem, const double *x, const double *y, const double *z,
                   const double *m, const double *a, const double *rc, double G, double Mstar,
                   double n1, int mode, int form, int n_big, double *acc)
{
    oracle_bs_acc_ml(n, mem, x, y, z, m, a, rc, G, Mstar, n1, mode, form, n_big, 0, 1, acc);
}

/*
 * Modified midpoint rule (Gragg) over a sub-step h with nsub steps of
 * H = h/nsub from y0 (f0 = f(y0)):
 *   z_0 = y0,  z_1 = z_0 + H f(z_0),  z_{k+1} = z_{k-1} + 2H f(z_k),
 *   result = (z_nsub + z_{nsub-1} + H f(z_nsub)) / 2,
 * whose error expands in even powers of H (what the extrapolation removes).
 */
static void bs_midpoint(const bs_group *g, const double *y0, const double *f0, double h, int nsub,
                        double *out, double *zp, double *zc, double *zn, double *fz)
{
    int L = 6 * g->n;
    double H = h / nsub;
    for (int q = 0; q < L; q++) { zp[q] = y0[q]; zc[q] = y0[q] + H * f0[q]; }
    for (int k = 1; k < nsub; k++) {
        bs_deriv(g, zc, fz);
        for (int q = 0; q < L; q++) zn[q] = zp[q] + 2.0 * H * fz[q];
        for (int q = 0; q < L; q++) { zp[q] = zc[q]; zc[q] = zn[q]; }
    }
    bs_deriv(g, zc, fz);
    for (int q = 0; q < L; q++) out[q] = 0.5 * (zc[q] + zp[q] + H * fz[q]);
}

#define BS_KMAX 8            /* extrapolation columns: midpoint step counts 2, 4, ..., 16 */
#define BS_GROW_COL 2        /* a sub-step accepted by column <= 2 doubles the next one */
#define BS_MIN_FRAC 0x1p-30  /* smallest sub-step, as a fraction of the drift */
#define BS_MAX_ATTEMPTS 4096 /* sub-step attempts per group and drift */

static int bs_n(int k) { return 2 * (k + 1); }

/*
 * Perfect mergers (Sect. 2: collisions are perfect mergers) after an accepted
 * sub-step: the first pair of members (in member order, i < j) that are not
 * ghosts and overlap, |x_i - x_j| < R_i + R_j, merges -- member i keeps the
 * total mass, the mass-weighted position and velocity and the radius
 * (R_i^3 + R_j^3)^(1/3) (equal density); member j becomes a ghost with m = 0,
 * R = 0 (m = -0.0: its state is kept, it exerts and feels no group force) -- and the
 * search repeats until no pair overlaps.  Returns the number of mergers.
 */
static int bs_merge(const bs_group *g, double *yv, double *m, double *R, int32_t *ghost)
{
    int merges = 0;
    for (;;) {
        int fi = -1, fj = -1;
        for (int i = 0; i < g->n && fi < 0; i++) {
            if (ghost[i]) continue;
            for (int j = i + 1; j < g->n; j++) {
                if (ghost[j]) continue;
                double dx = yv[6 * j] - yv[6 * i], dy = yv[6 * j + 1] - yv[6 * i + 1];
                double dz = yv[6 * j + 2] - yv[6 * i + 2];
                double rr = R[g->mem[i]] + R[g->mem[j]];
                if (dx * dx + dy * dy + dz * dz < rr * rr) { fi = i; fj = j; break; }
            }
        }
        if (fi < 0) return merges;
        int bi = g->mem[fi], bj = g->mem[fj];
        double mi = m[bi], mj = m[bj], mt = mi + mj;
        for (int c = 0; c < 6; c++) {
            double u = yv[6 * fi + c], w = yv[6 * fj + c];
            yv[6 * fi + c] = (mt > 0.0) ? (mi * u + mj * w) / mt : 0.5 * (u + w);
        }
        m[bi] = mt;
        R[bi] = cbrt(R[bi] * R[bi] * R[bi] + R[bj] * R[bj] * R[bj]);
        m[bj] = -0.0;                   /* the ghost mark: numerically zero, sign bit set */
        R[bj] = 0.0;
        ghost[fj] = 1;
        merges++;
    }
}

/*
 * Bulirsch-Stoer integration of one group over dt (Stoer & Bulirsch,
 * Introduction to Numerical Analysis, Sect. 7.2.14): each sub-step h runs the
 * modified midpoint rule with n_k = 2, 4, ..., 16 steps and extrapolates the
 * results to H -> 0 with the Aitken-Neville scheme in H^2,
 *   T[k][j] = T[k][j-1] + (T[k][j-1] - T[k-1][j-1]) * n_{k-j}^2 / (n_k^2 - n_{k-j}^2).
 * Column k (k >= 1) is accepted when, for every member,
 *   max_c |T[k][k] - T[k][k-1]| <= tol * |x| (position) and tol * |v| (velocity)
 * (norms of the member's state at the start of the sub-step; 1 where zero).
 * The first sub-step is the largest binary fraction f of dt for which no
 * interacting pair moves by more than its separation (f |dt| |v_ij| <= r_ij).
 * A sub-step with no accepted column is halved; one accepted at a column
 * <= BS_GROW_COL doubles the next.  Sub-steps are fractions of dt; a sub-step
 * at BS_MIN_FRAC is accepted at the last column anyway, and after
 * BS_MAX_ATTEMPTS attempts the members drift the rest of dt on their Kepler
 * orbits (both count as forced).  With radii R (per
 * body, NULL: no collisions) overlapping members merge after every accepted
 * sub-step (bs_merge); the absorbed bodies get dead[b] = 1 (per body, needed
 * with R), m = R = 0.  Updates the members' entries of x..vz, m, R; returns 1
 * if an acceptance was forced, else 0; *merges (optional) accumulates the
 * mergers.
 */
static int bs_group_run(int n, const int32_t *mem, double *x, double *y, double *z,
                        double *vx, double *vy, double *vz, double *m, const double *a,
                        const double *rc, double *R, int32_t *dead, double G, double Mstar,
                        double n1, int mode, int form, int n_big, double dt, double tol,
                        int *merges, int nlev, int nsub, int *accepted, int *attempts)
{
    int32_t *ghost = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    bs_group g = {n, mem, m, a, rc, G, Mstar, n1, mode, form, n_big, ghost, nlev, nsub};
    int L = 6 * n;
    double *buf = (double *)malloc(sizeof(double) * (size_t)L * (7 + BS_KMAX * BS_KMAX));
    double *yv = buf, *f0 = yv + L, *zp = f0 + L, *zc = zp + L, *zn = zc + L, *fz = zn + L,
           *sc = fz + L, *T = sc + L;       /* T[(k * BS_KMAX + j) * L + q] */
    for (int k = 0; k < n; k++) {
        int b = mem[k];
        double *s = yv + 6 * k;
        s[0] = x[b]; s[1] = y[b]; s[2] = z[b]; s[3] = vx[b]; s[4] = vy[b]; s[5] = vz[b];
    }
    double done = 0.0, frac = 1.0;           /* fractions of dt: exact binary values */
    int forced = 0, nmerge = 0;
    /* first sub-step: the largest binary fraction f of dt with f |dt| |v_ij| <= |x_ij|
       for every interacting pair (no pair crosses more than its separation in it) */
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            if (tp_pair(n_big, mem[i], mem[j])) continue;
            const double *si = yv + 6 * i, *sj = yv + 6 * j;
            double dx = sj[0] - si[0], dy = sj[1] - si[1], dz = sj[2] - si[2];
            double ux = sj[3] - si[3], uy = sj[4] - si[4], uz = sj[5] - si[5];
            double r2 = dx * dx + dy * dy + dz * dz, v2 = ux * ux + uy * uy + uz * uz;
            double f = 1.0;
            while (f > BS_MIN_FRAC && (f * fabs(dt)) * (f * fabs(dt)) * v2 > r2) f *= 0.5;
            if (f < frac) frac = f;
        }
    }
    int n_acc = 0, n_att = 0;
    for (int att = 0; att < BS_MAX_ATTEMPTS && done < 1.0; att++) {
        double h = frac * dt;
        n_att++;
        for (int k = 0; k < n; k++) {        /* error scales of this sub-step */
            const double *s = yv + 6 * k;
            double px = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            double pv = sqrt(s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
            sc[6 * k] = px > 0.0 ? px : 1.0;
            sc[6 * k + 3] = pv > 0.0 ? pv : 1.0;
        }
        bs_deriv(&g, yv, f0);
        int acc_col = -1;
        for (int k = 0; k < BS_KMAX; k++) {
            double *Tk0 = T + (size_t)(k * BS_KMAX) * L;
            bs_midpoint(&g, yv, f0, h, bs_n(k), Tk0, zp, zc, zn, fz);
            for (int j = 1; j <= k; j++) {
                double nk = bs_n(k), nkj = bs_n(k - j);
                double cf = (nkj * nkj) / (nk * nk - nkj * nkj);
                double *Tkj = T + (size_t)(k * BS_KMAX + j) * L;
                const double *Tkj1 = T + (size_t)(k * BS_KMAX + j - 1) * L;
                const double *Tk1j1 = T + (size_t)((k - 1) * BS_KMAX + j - 1) * L;
                for (int q = 0; q < L; q++) Tkj[q] = Tkj1[q] + (Tkj1[q] - Tk1j1[q]) * cf;
            }
            if (k == 0) continue;
            const double *Tkk = T + (size_t)(k * BS_KMAX + k) * L;
            const double *Tkm = T + (size_t)(k * BS_KMAX + k - 1) * L;
            double err = 0.0;
            for (int q = 0; q < L; q++) {
                double e = fabs(Tkk[q] - Tkm[q]) / sc[6 * (q / 6) + ((q % 6) < 3 ? 0 : 3)];
                if (e > err) err = e;
            }
            if (err <= tol) { acc_col = k; break; }
        }
        if (acc_col < 0 && frac <= BS_MIN_FRAC) {
            acc_col = BS_KMAX - 1;              /* forced: keep the last column */
            forced = 1;
        }
        if (acc_col < 0) { frac *= 0.5; continue; }
        const double *Tacc = T + (size_t)(acc_col * BS_KMAX + acc_col) * L;
        for (int q = 0; q < L; q++) yv[q] = Tacc[q];
        if (R) nmerge += bs_merge(&g, yv, m, R, ghost);
        n_acc++;
        done += frac;
        if (acc_col <= BS_GROW_COL) frac *= 2.0;
        if (frac > 1.0 - done) frac = 1.0 - done;
    }
    if (done < 1.0) {   /* out of attempts: the rest of the drift on Kepler orbits (level 0) */
        forced = 1;
        for (int k = 0; k < n; k++) oracle_kepler(G * Mstar, yv + 6 * k, (1.0 - done) * dt, 50);
    }
    for (int k = 0; k < n; k++) {
        int b = mem[k];
        const double *s = yv + 6 * k;
        x[b] = s[0]; y[b] = s[1]; z[b] = s[2]; vx[b] = s[3]; vy[b] = s[4]; vz[b] = s[5];
        if (ghost[k] && dead) dead[b] = 1;
    }
    if (merges) *merges += nmerge;
    if (accepted) *accepted = n_acc;
    if (attempts) *attempts = n_att;
    free(buf);
    free(ghost);
    return forced;
}

int oracle_bs_group_full(int n, const int32_t *mem, double *x, double *y, double *z,
                         double *vx, double *vy, double *vz, double *m, const double *a,
                         const double *rc, double *R, int32_t *dead, double G, double Mstar,
                         double n1, int mode, int form, int n_big, double dt, double tol,
                         int *merges)
{
    return bs_group_run(n, mem, x, y, z, vx, vy, vz, m, a, rc, R, dead, G, Mstar, n1, mode, form, n_big,
                        dt, tol, merges, 0, 1, NULL, NULL);
}

/* oracle_bs_group without collisions, also reporting the accepted sub-steps
 * and the attempts of the step-size control. */
int oracle_bs_group_counted(int n, const int32_t *mem, double *x, double *y, double *z,
                            double *vx, double *vy, double *vz, const double *m, const double *a,
                            const double *rc, double G, double Mstar, double n1, int mode, int form,
                            int n_big, double dt, double tol, int *accepted, int *attempts)
{
    return bs_group_run(n, mem, x, y, z, vx, vy, vz, (double *)m, a, rc, NULL, NULL, G, Mstar, n1, mode, form,
                        n_big, dt, tol, NULL, 0, 1, accepted, attempts);
}

/* oracle_bs_group_full without collisions. */
int oracle_bs_group(int n, const int32_t *mem, double *x, double *y, double *z,
                    double *vx, double *vy, double *vz, const double *m, const double *a,
                    const double *rc, double G, double Mstar, double n1, int mode, int form,
                    int n_big, double dt, double tol)
{
    return oracle_bs_group_full(n, mem, x, y, z, vx, vy, vz, (double *)m, a, rc, NULL, NULL, G, Mstar,
                                n1, mode, form, n_big, dt, tol, NULL);
}

/*
 * The intermediate levels (Sect. 1).  ml_level(l, group, T) moves a group of
 * level l (1 <= l <= L) over T in s sub-steps of h = T / s, each
 *   kick(h/2):  v_i += h/2 sum_{j in group} G m_j W_l(r_ij) (x_j - x_i) / r_ij^3
 *   drift(h):   subgroups = connected components of the member pairs with
 *               r_ij < r_crit,l, and of the pairs with r_crit,l <= r_ij <
 *               1.5 r_crit,l whose straight-line relative motion over h
 *               enters r_crit,l (the level's predicted entries, as in the
 *               step's first kick); members outside every subgroup take the
 *               Kepler drift over h, each subgroup (in order of its smallest
 *               body) moves on level l + 1 over h -- the Bulirsch-Stoer
 *               integrator with W_{L+1} once l = L
 *   kick(h/2)
 * Members are in ascending body order, every sum in that order.  Ghosts
 * (m = -0.0, from mergers in a Bulirsch-Stoer subgroup) feel and exert no
 * level force, join no subgroup and keep the Kepler drift.  Comparisons of
 * squares, as written, without contraction.
 */
typedef struct {
    double *x, *y, *z, *vx, *vy, *vz, *m, *R;
    const double *a, *rc;
    int32_t *dead;
    double G, Mstar, n1, tol;
    int mode, form, n_big, L, s, max_iter;
    int forced, merges, bad;
} ml_ctx;

/* The level-l share of the pair forces on each member of a group (ascending
 * body indices), without the central term: acc[3k + c] for member k,
 *   sum_{j in group} G m_j W_l(r_kj) (x_j - x_k) / r_kj^3
 * (ghosts and pairs of two test particles excluded). */
void oracle_ml_level_acc(int n, const int32_t *mem, const double *x, const double *y, const double *z,
                         const double *m, const double *a, const double *rc, double G, double Mstar, double n1,
                         int mode, int form, int n_big, int l, int L, int s, double *acc)
{
    for (int i = 0; i < n; i++) {
        int bi = mem[i];
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (!signbit(m[bi])) {
            for (int j = 0; j < n; j++) {
                int bj = mem[j];
                if (j == i || signbit(m[bj]) || tp_pair(n_big, bi, bj)) continue;
                double dx = x[bj] - x[bi], dy = y[bj] - y[bi], dz = z[bj] - z[bi];
                double q2 = dx * dx + dy * dy + dz * dz;
                if (q2 == 0.0) continue;
                double q = sqrt(q2);
                double rcij = oracle_pair_rcrit(mode, m[bi], m[bj], a[bi], a[bj], rc[bi], rc[bj], n1, Mstar);
                if (q >= rcij) continue;                  /* W_l = 0 outside r_crit,0 */
                double f = G * m[bj] * oracle_ml_weight(q, rcij, l, L, s, form) / (q2 * q);
                ax += f * dx;
                ay += f * dy;
                az += f * dz;
            }
        }
        acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az;
    }
}

static void ml_kick(ml_ctx *c, int l, int n, const int32_t *mem, double tau)
{
    double *acc = (double *)calloc((size_t)(3 * n > 0 ? 3 * n : 1), sizeof(double));
    oracle_ml_level_acc(n, mem, c->x, c->y, c->z, c->m, c->a, c->rc, c->G, c->Mstar, c->n1, c->mode, c->form,
                        c->n_big, l, c->L, c->s, acc);
    for (int i = 0; i < n; i++) {
        int bi = mem[i];
        c->vx[bi] += tau * acc[3 * i];
        c->vy[bi] += tau * acc[3 * i + 1];
        c->vz[bi] += tau * acc[3 * i + 2];
    }
    free(acc);
}

/* Is (bi, bj) a pair of the subgroups of level l + 1 for a drift of h? */
static int subpair(const double *x, const double *y, const double *z, const double *vx, const double *vy,
                   const double *vz, const double *m, const double *a, const double *rc, double n1, double Mstar,
                   int mode, int n_big, int l, int s, int bi, int bj, double h)
{
    if (signbit(m[bi]) || signbit(m[bj]) || tp_pair(n_big, bi, bj)) return 0;
    double dx = x[bj] - x[bi], dy = y[bj] - y[bi], dz = z[bj] - z[bi];
    double q2 = dx * dx + dy * dy + dz * dz;
    double rcij = oracle_pair_rcrit(mode, m[bi], m[bj], a[bi], a[bj], rc[bi], rc[bj], n1, Mstar);
    double rcl = oracle_ml_radius(rcij, l, s);
    double rcl2 = rcl * rcl, rout = 1.5 * rcl;
    if (q2 < rcl2) return 1;
    if (q2 >= rout * rout) return 0;
    double ux = vx[bj] - vx[bi], uy = vy[bj] - vy[bi], uz = vz[bj] - vz[bi];
    double uu = ux * ux + uy * uy + uz * uz, du = dx * ux + dy * uy + dz * uz;
    double tlo = h < 0.0 ? h : 0.0, thi = h < 0.0 ? 0.0 : h;
    double t = uu > 0.0 ? -du / uu : 0.0;
    if (t < tlo) t = tlo;
    if (t > thi) t = thi;
    double px = dx + ux * t, py = dy + uy * t, pz = dz + uz * t;
    return px * px + py * py + pz * pz < rcl2;
}

static int ml_subpair(const ml_ctx *c, int l, int bi, int bj, double h)
{
    return subpair(c->x, c->y, c->z, c->vx, c->vy, c->vz, c->m, c->a, c->rc, c->n1, c->Mstar, c->mode, c->n_big,
                   l, c->s, bi, bj, h);
}

/* The member pairs (i < j, member order) of a level-l group that form the
 * subgroups of level l + 1 for a drift of h: inside r_crit,l, or within
 * 1.5 r_crit,l and entering r_crit,l on their straight-line relative motion
 * within h.  Writes at most `cap` pairs of body indices; returns the count. */
int64_t oracle_ml_subpairs(int n, const int32_t *mem, const double *x, const double *y, const double *z,
                           const double *vx, const double *vy, const double *vz, const double *m, const double *a,
                           const double *rc, double n1, double Mstar, int mode, int n_big, int l, int s, double h,
                           int32_t *pairs, int64_t cap)
{
    int64_t cnt = 0;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            if (!subpair(x, y, z, vx, vy, vz, m, a, rc, n1, Mstar, mode, n_big, l, s, mem[i], mem[j], h)) continue;
            if (cnt < cap) { pairs[2 * cnt] = mem[i]; pairs[2 * cnt + 1] = mem[j]; }
            cnt++;
        }
    return cnt;
}

static void ml_level(ml_ctx *c, int l, int n, const int32_t *mem, double T)
{
    double h = T / c->s;
    int32_t *root = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *inpair = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *sub = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int step = 0; step < c->s; step++) {
        ml_kick(c, l, n, mem, 0.5 * h);
        for (int i = 0; i < n; i++) { root[i] = i; inpair[i] = 0; }
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) {
                if (!ml_subpair(c, l, mem[i], mem[j], h)) continue;
                inpair[i] = inpair[j] = 1;
                int ri = uf_root(root, i), rj = uf_root(root, j);
                if (ri < rj) root[rj] = ri;
                else if (rj < ri) root[ri] = rj;
            }
        for (int i = 0; i < n; i++) {
            if (inpair[i]) continue;
            int b = mem[i];
            double st[6] = {c->x[b], c->y[b], c->z[b], c->vx[b], c->vy[b], c->vz[b]};
            c->bad += oracle_kepler(c->G * c->Mstar, st, h, c->max_iter);
            c->x[b] = st[0]; c->y[b] = st[1]; c->z[b] = st[2];
            c->vx[b] = st[3]; c->vy[b] = st[4]; c->vz[b] = st[5];
        }
        for (int r = 0; r < n; r++) {
            if (!inpair[r] || uf_root(root, r) != r) continue;
            int cnt = 0;
            for (int k = r; k < n; k++)
                if (inpair[k] && uf_root(root, k) == r) sub[cnt++] = mem[k];
            if (l < c->L)
                ml_level(c, l + 1, cnt, sub, h);
            else
                c->forced += bs_group_run(cnt, sub, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->m, c->a, c->rc, c->R,
                                          c->dead, c->G, c->Mstar, c->n1, c->mode, c->form, c->n_big, h, c->tol,
                                          &c->merges, c->L, c->s, NULL, NULL);
        }
        ml_kick(c, l, n, mem, 0.5 * h);
    }
    free(root);
    free(inpair);
    free(sub);
}

/* One group of the step's drift on level 1 with L >= 1 intermediate levels and
 * s sub-steps per level (members in ascending order).  Returns 1 if a
 * Bulirsch-Stoer acceptance was forced; *merges, *bad (optional) accumulate
 * the mergers and the Kepler solves that hit the cap. */
int oracle_ml_group(int n, const int32_t *mem, double *x, double *y, double *z,
                    double *vx, double *vy, double *vz, double *m, const double *a,
                    const double *rc, double *R, int32_t *dead, double G, double Mstar,
                    double n1, int mode, int form, int n_big, double dt, double tol,
                    int nlev, int nsub, int max_iter, int *merges, int *bad)
{
    ml_ctx c = {x, y, z, vx, vy, vz, m, R, a, rc, dead, G, Mstar, n1, tol, mode, form, n_big, nlev, nsub,
                max_iter, 0, 0, 0};
    ml_level(&c, 1, n, mem, dt);
    if (merges) *merges += c.merges;
    if (bad) *bad += c.bad;
    return c.forced > 0 ? 1 : 0;
}

/*
 * Drift of the hybrid step with the close-encounter level: HC(dt/2); every
 * body outside the groups of `pairs` (the encounter pairs of the step's
 * first kick; pairs with a dead body do not count) on its Kepler orbit, every
 * group by oracle_bs_group_full (a, rc from that kick; mergers when R is
 * given), or with nlev >= 1 intermediate levels of nsub sub-steps by
 * oracle_ml_group; HC(dt/2); then removal: a body still alive with |x|^2 < r_in^2 or
 * |x|^2 > r_out^2 (each test off when its radius is <= 0) becomes dead with
 * m = 0 (and R = 0).  dead (per body) is needed with R or the radii.
 * Returns the number of Kepler solves that hit the cap; *bs_forced and
 * *merges (optional) get the groups with a forced Bulirsch-Stoer acceptance
 * and the mergers.
 */
int oracle_drift_groups_ml(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                           double *m, const double *a, const double *rc, double *R, int32_t *dead,
                           int64_t npairs, const int32_t *pairs, double G, double Mstar, double n1,
                           int mode, int form, int n_big, double dt, double tol, int max_iter,
                           double r_in, double r_out, int nlev, int nsub, int *bs_forced, int *merges)
{
    int bad = 0, forced = 0, nmerge = 0;
    size_t n = (size_t)(N > 0 ? N : 1);
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *live = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(npairs > 0 ? npairs : 1));
    int64_t nlive = 0;
    for (int64_t p = 0; p < npairs; p++) {
        if (dead && (dead[pairs[2 * p]] || dead[pairs[2 * p + 1]])) continue;
        live[2 * nlive] = pairs[2 * p];
        live[2 * nlive + 1] = pairs[2 * p + 1];
        nlive++;
    }
    oracle_groups(N, nlive, live, label);
    oracle_hc_drift(N, x, y, z, vx, vy, vz, m, Mstar, 0.5 * dt);
    #pragma omp parallel for reduction(+:bad)
    for (int i = 0; i < N; i++) {
        if (label[i] >= 0) continue;
        double s[6] = {x[i], y[i], z[i], vx[i], vy[i], vz[i]};
        bad += oracle_kepler(G * Mstar, s, dt, max_iter);
        x[i] = s[0]; y[i] = s[1]; z[i] = s[2];
        vx[i] = s[3]; vy[i] = s[4]; vz[i] = s[5];
    }
    for (int r = 0; r < N; r++) {
        if (label[r] != r) continue;         /* r is the smallest member of its group */
        int cnt = 0;
        for (int v = r; v < N; v++)
            if (label[v] == r) mem[cnt++] = v;
        if (nlev > 0)
            forced += oracle_ml_group(cnt, mem, x, y, z, vx, vy, vz, m, a, rc, R, dead, G, Mstar, n1, mode, form,
                                      n_big, dt, tol, nlev, nsub, max_iter, &nmerge, &bad);
        else
            forced += oracle_bs_group_full(cnt, mem, x, y, z, vx, vy, vz, m, a, rc, R, dead, G, Mstar, n1,
                                           mode, form, n_big, dt, tol, &nmerge);
    }
    oracle_hc_drift(N, x, y, z, vx, vy, vz, m, Mstar, 0.5 * dt);
    if (dead && (r_in > 0.0 || r_out > 0.0)) {
        for (int i = 0; i < N; i++) {
            if (dead[i]) continue;
            double r2 = x[i] * x[i] + y[i] * y[i] + z[i] * z[i];
            if ((r_in > 0.0 && r2 < r_in * r_in) || (r_out > 0.0 && r2 > r_out * r_out)) {
                dead[i] = 1;
                m[i] = -0.0;
                if (R) R[i] = 0.0;
            }
        }
    }
    if (bs_forced) *bs_forced = forced;
    if (merges) *merges += nmerge;
    free(label);
    free(mem);
    free(live);
    return bad;
}

/* oracle_drift_groups_ml without intermediate levels. */
int oracle_drift_groups_full(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                             double *m, const double *a, const double *rc, double *R, int32_t *dead,
                             int64_t npairs, const int32_t *pairs, double G, double Mstar, double n1,
                             int mode, int form, int n_big, double dt, double tol, int max_iter,
                             double r_in, double r_out, int *bs_forced, int *merges)
{
    return oracle_drift_groups_ml(N, x, y, z, vx, vy, vz, m, a, rc, R, dead, npairs, pairs, G, Mstar, n1, mode,
                                  form, n_big, dt, tol, max_iter, r_in, r_out, 0, 1, bs_forced, merges);
}

/* oracle_drift_groups_full without collisions or removal. */
int oracle_drift_groups(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                        const double *m, const double *a, const double *rc,
                        int64_t npairs, const int32_t *pairs, double G, double Mstar, double n1,
                        int mode, int form, int n_big, double dt, double tol, int max_iter,
                        int *bs_forced)
{
    return oracle_drift_groups_full(N, x, y, z, vx, vy, vz, (double *)m, a, rc, NULL, NULL, npairs, pairs,
                                    G, Mstar, n1, mode, form, n_big, dt, tol, max_iter, 0.0, 0.0,
                                    bs_forced, NULL);
}

/*
 * Hybrid step with the close-encounter level, repeated nsteps times:
 * r_crit, the encounter pairs and the predicted entries of the state,
 * kick(dt/2), the drift of oracle_drift_groups_ml on both lists (nlev
 * intermediate levels of nsub sub-steps; mergers
 * with R, removal with r_in / r_out, dead flags per body), kick(dt/2).  Returns the Kepler cap count; *bs_forced and
 * *merges (optional) accumulate the forced Bulirsch-Stoer acceptances and the
 * mergers.
 */
int oracle_step_ml(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                   double *m, double *R, int32_t *dead, double G, double Mstar, double dt, double n1,
                   double n2, int mode, int form, int n_big, int max_iter, double tol, double r_in,
                   double r_out, int nlev, int nsub, int nsteps, int *bs_forced, int *merges)
{
    int bad = 0, forced = 0;
    size_t n = (size_t)(N > 0 ? N : 1);
    double *ax = (double *)malloc(sizeof(double) * n);
    double *ay = (double *)malloc(sizeof(double) * n);
    double *az = (double *)malloc(sizeof(double) * n);
    double *a = (double *)malloc(sizeof(double) * n);
    double *rc = (double *)malloc(sizeof(double) * n);
    int64_t cap = 16 * (int64_t)n;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cap);
    for (int s = 0; s < nsteps; s++) {
        oracle_rcrit(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, a, rc);
        int64_t np = oracle_encounters(N, x, y, z, m, a, rc, n1, Mstar, mode, n_big, pairs, cap,
                                       0.0, NULL, 0, NULL);
        if (np > cap) {                       /* grow and list again */
            free(pairs);
            cap = np;
            pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cap);
            np = oracle_encounters(N, x, y, z, m, a, rc, n1, Mstar, mode, n_big, pairs, cap,
                                   0.0, NULL, 0, NULL);
        }
        /* the drift's groups: the encounter pairs and the predicted entries */
        int64_t npr = oracle_predicted_pairs(N, x, y, z, vx, vy, vz, m, a, rc, n1, Mstar, mode, n_big, dt,
                                             pairs + 2 * np, cap - np);
        if (np + npr > cap) {
            int32_t *bigger = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(np + npr));
            for (int64_t q = 0; q < 2 * np; q++) bigger[q] = pairs[q];
            free(pairs);
            pairs = bigger;
            cap = np + npr;
            oracle_predicted_pairs(N, x, y, z, vx, vy, vz, m, a, rc, n1, Mstar, mode, n_big, dt,
                                   pairs + 2 * np, npr);
        }
        oracle_kick(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, mode, form, n_big, 0.5 * dt, ax, ay, az);
        int f = 0;
        bad += oracle_drift_groups_ml(N, x, y, z, vx, vy, vz, m, a, rc, R, dead, np + npr, pairs, G, Mstar, n1,
                                      mode, form, n_big, dt, tol, max_iter, r_in, r_out, nlev, nsub, &f, merges);
        forced += f;
        oracle_kick(N, x, y, z, vx, vy, vz, m, G, Mstar, dt, n1, n2, mode, form, n_big, 0.5 * dt, ax, ay, az);
    }
    if (bs_forced) *bs_forced += forced;
    free(ax); free(ay); free(az); free(a); free(rc); free(pairs);
    return bad;
}

/* oracle_step_ml without intermediate levels. */
int oracle_step_full(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                     double *m, double *R, int32_t *dead, double G, double Mstar, double dt, double n1,
                     double n2, int mode, int form, int n_big, int max_iter, double tol, double r_in,
                     double r_out, int nsteps, int *bs_forced, int *merges)
{
    return oracle_step_ml(N, x, y, z, vx, vy, vz, m, R, dead, G, Mstar, dt, n1, n2, mode, form, n_big, max_iter,
                          tol, r_in, r_out, 0, 1, nsteps, bs_forced, merges);
}

/* oracle_step_full without collisions or removal. */
int oracle_step_bs(int N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                   const double *m, double G, double Mstar, double dt, double n1, double n2,
                   int mode, int form, int n_big, int max_iter, double tol, int nsteps, int *bs_forced)
{
    return oracle_step_full(N, x, y, z, vx, vy, vz, (double *)m, NULL, NULL, G, Mstar, dt, n1, n2, mode, form,
                            n_big, max_iter, tol, 0.0, 0.0, nsteps, bs_forced, NULL);
}

/* ------------------------------------- energy and angular momentum -------- */

/*
 * out[0] = E = sum m v^2/2 + |P|^2/(2 M*) - sum G M* m_i / r_i
 *              - sum_{i<j} G m_i m_j / r_ij     (democratic-heliocentric H;
 *                test-particle pairs excluded when n_big >= 0)
 * out[1..3] = L = sum m_i x_i x v_i.
 */
void oracle_energy(int N, const double *x, const double *y, const double *z,
                   const double *vx, const double *vy, const double *vz, const double *m,
                   double G, double Mstar, int n_big, double *out)
{
    nsum e = {0, 0}, lx = {0, 0}, ly = {0, 0}, lz = {0, 0};
    double P[3];
    oracle_momentum(N, vx, vy, vz, m, P);
    nadd(&e, (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * Mstar));
    for (int i = 0; i < N; i++) {
        double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
        nadd(&e, 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]));
        nadd(&e, -G * Mstar * m[i] / r);
        nadd(&lx, m[i] * (y[i] * vz[i] - z[i] * vy[i]));
        nadd(&ly, m[i] * (z[i] * vx[i] - x[i] * vz[i]));
        nadd(&lz, m[i] * (x[i] * vy[i] - y[i] * vx[i]));
    }
    for (int i = 0; i < N; i++) {
        for (int j = i + 1; j < N; j++) {
            if (tp_pair(n_big, i, j)) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            nadd(&e, -G * m[i] * m[j] / sqrt(dx * dx + dy * dy + dz * dz));
        }
    }
    out[0] = nval(&e);
    out[1] = nval(&lx); out[2] = nval(&ly); out[3] = nval(&lz);
}
